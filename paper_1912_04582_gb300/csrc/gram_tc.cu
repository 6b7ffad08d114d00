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
// Tensor-core mapping.  Slice k is stored as the bf16 value s_k 2^-7k (exact: a small
// integer times a power of two, formed by rounding at level k directly), so the
// accumulator of slice product (k, l) holds 2^-7(k+l) D^(k,l), still exact.  The slices
// of a K-chunk of 64 columns sit in shared memory one after the other, sp = n rounded
// up to 8 rows each, as a K-major 128-byte swizzled bf16 operand.  One MMA group takes 128 consecutive rows as A (the M = 128
// accumulator lanes hold several slices) and a run of rows as B (N up to 256
// columns hold several slices): a single instruction forms up to 4 x 5 slice
// products.  One to three groups cover every needed pair for n <= 64; their FP32
// accumulators live in tensor memory (TMEM).  Per CTA (persistent, one per SM): one
// thread streams the cell's K-chunks by 2-D TMA loads (cp.async.bulk.tensor) into a
// four-deep ring, once when the row maxima are given (the assembly of X records them),
// else twice (row scales, then slicing); eight warps slice each chunk into
// one of three bf16 stages while the tensor cores work on the previous ones (one
// mbarrier per stage signalled by tcgen05.commit), and one of their threads issues
// the MMAs.  After a cell's last chunk the accumulators are read back (tcgen05.ld)
// tile by tile and combined while the next cell's chunks already load.  Every wait
// is bounded: on timeout the CTA sets bit 1 of *flag, drains its loads and MMAs,
// frees its tensor memory and returns.
#include <cuda.h>

#include <cstdint>
#include <mutex>

#include "dvm_internal.h"
#include "tucker.h"

namespace dvm {
namespace {

constexpr int kTcMaxStages = 3;     // shared-memory stages of sliced chunks (at most)
constexpr int kTcLevels = 2 * kTcSlices - 2;  // slice-product levels k + l = 0 .. 7
constexpr int kTcKC = 64;              // columns per chunk: one 128-byte bf16 row
constexpr int kTcRowBytes = 128;
constexpr int kTcRawStages = 4;              // TMA ring of FP32 chunks
constexpr int kTcRawBytes = 64 * kTcKC * 4;  // one chunk of up to 64 rows
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

// bf16 of two floats with at most 8 significant bits (small integers times powers of
// two), packed (lo in the low half): such a float has zero low 16 bits, so its bf16 is
// its upper half, taken by a byte permute
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// 1.5 * 2^(23 - 7k): adding and removing it rounds to a multiple of 2^-7k
__device__ constexpr float kSliceMagic[kTcSlices] = {12582912.0f, 98304.0f, 768.0f, 6.0f,
                                                     0.046875f};

// 2^7m: an accumulator of level m holds 2^-7m times an integer
__device__ constexpr float kLevelScale[kTcLevels] = {1.0f, 128.0f, 16384.0f, 2097152.0f,
                                                     268435456.0f, 34359738368.0f,
                                                     4398046511104.0f, 562949953421312.0f};

// paired FP32 arithmetic (two lanes of a 64-bit register), round to nearest
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

}  // namespace

// Plan of the MMA groups for one row count n (host-side; see GramTcPlan in tucker.h):
// the set of at most three groups (A = slices a0 .. a0 + na - 1 in the 128 accumulator
// lanes, B = slices b0 .. b0 + nb - 1 in at most 256 columns) that forms every needed
// slice product with the fewest tensor-memory columns (the MMA work is proportional to
// them), found by exhaustive search; each product is owned by the first group that
// forms it.
// offset of row a in the packed upper triangle of an n x n matrix (row a: entries (a, a..n-1))
__host__ __device__ inline int tri_row(int n, int a) { return a * n - ((a * (a - 1)) >> 1); }

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
  // three stages of sliced chunks where they fit beside the TMA ring and the level
  // accumulators in 227 KB of shared memory, else two (n > 56)
  const size_t fixed = 1024 + (size_t)kTcRawStages * kTcRawBytes +
                       sizeof(int) * kTcLevels * (size_t)(n * (n + 1) / 2) + 1024;
  p.nstages = fixed + (size_t)kTcMaxStages * p.buf_rows * kTcRowBytes <= 227 * 1024
                  ? kTcMaxStages
                  : kTcMaxStages - 1;
  p.ltri = n * (n + 1) / 2;  // level accumulators: the packed upper triangle
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

// level accumulators: int32 [kTcLevels][ltri]
static size_t level_bytes(const GramTcPlan &p) { return sizeof(int) * kTcLevels * (size_t)p.ltri; }

static size_t smem_for(const GramTcPlan &p, int nstages) {
  const size_t stages = (size_t)nstages * p.buf_rows * kTcRowBytes;
  const size_t raw = (size_t)kTcRawStages * kTcRawBytes;
  return 1024 + stages + raw + level_bytes(p) + 64 * (2 * sizeof(int) + sizeof(float)) + 64;
}

size_t gram_tc_smem_bytes(const GramTcPlan &p) { return smem_for(p, p.nstages); }

namespace {

constexpr int kTcConsumers = 384;                  // twelve slicing warps
constexpr int kTcThreadsAll = kTcConsumers + 64;   // plus the TMA producer and MMA warps

struct TcArgs {
  int64_t ncell;
  int K;
  float2 *C;        // cell j: C + j * cstride, n x n double-float pairs (hi, lo), or
  double *Cd;       // the same as doubles (exactly one of C, Cd is set)
  int64_t cstride;
  double *disc;     // [ncell] set to 0 (no columns left out), may be null
  int *flag;
  const float *rowmax;  // cell j: rowmax + j * rstride, each row's largest |x| (or null:
  int64_t rstride;      // then a first pass over X finds them)
  long long *phase;     // optional per-role cycle counters, slots 16-26 (null: off)
  GramTcPlan plan;
};

// cycles of one role's lane, accumulated into phase[slot] when phase is set; no effect on
// the computation
struct RoleClock {
  long long *acc;
  long long t;
  __device__ explicit RoleClock(long long *a) {
    acc = a;
    t = a ? (long long)clock64() : 0;
  }
  __device__ __forceinline__ void mark(int slot) {
    if (!acc) return;
    const long long now = (long long)clock64();
    atomicAdd(reinterpret_cast<unsigned long long *>(acc + slot), (unsigned long long)(now - t));
    t = now;
  }
  __device__ __forceinline__ void reset() {
    if (acc) t = (long long)clock64();
  }
};

// bounded wait on one mbarrier phase that also gives up once *abort is set
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, const volatile int *abort) {
  uint32_t done = 0;
  for (int it = 0; it < kTcWaitIters && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (!done && *abort) break;
  }
  return done != 0;
}

// barrier of the eight consumer warps (named barrier 1) returning the AND of v
__device__ __forceinline__ bool consumers_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kTcConsumers)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTcConsumers) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 2-D tiled TMA load of one chunk (x: column, y: row) completing on bar
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, int x, int y,
                                         uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Warp roles.  Warp 0: tensor-memory allocation and, in lane 0, the TMA producer: for
// each of the CTA's cells, the cell's K-chunks (n rows x 64 columns of FP32, one 2-D
// tiled load each; twice when the row maxima are not given) into a four-deep ring whose
// slots the slicing warps release.  Warp 1, lane 0: the MMA issuer: waits until the
// slicing warps have filled a stage, issues the stage's MMAs and commits them to the
// stage's "freed" barrier (and, after a cell's last chunk, to the "accumulators full"
// barrier); before a cell's first chunk it waits until the previous cell's
// accumulators have been read.  Warps 2-13: the slicing warps: row scales, slicing of
// each chunk into a free stage, and the read-back and combination of the accumulators.
// No CTA-wide barrier is taken per chunk: every hand-off is an mbarrier.
template <bool kTimed>
__global__ void __launch_bounds__(kTcThreadsAll, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap xmap, TcArgs A) {
  extern __shared__ unsigned char tc_raw[];
  const GramTcPlan &P = A.plan;
  const int n = P.n, sp = P.sp, K = A.K;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  const size_t stage_bytes = (size_t)P.buf_rows * kTcRowBytes;  // a multiple of 1024
  const uint32_t NS = (uint32_t)P.nstages;
  const int ntri = n * (n + 1) / 2, ltri = P.ltri;
  unsigned char *stages = base;
  unsigned char *raw = stages + NS * stage_bytes;
  // exact integer sums of the slice products per level k + l, upper triangle
  int *Lacc = reinterpret_cast<int *>(raw + kTcRawStages * kTcRawBytes);
  int *rexp = Lacc + kTcLevels * ltri;
  float *rinv = reinterpret_cast<float *>(rexp + 64);

  __shared__ __align__(8) unsigned long long s_full[kTcRawStages], s_empty[kTcRawStages];
  __shared__ __align__(8) unsigned long long s_ready[kTcMaxStages], s_freed[kTcMaxStages];
  __shared__ __align__(8) unsigned long long s_accf, s_acce;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  constexpr int kWarpsC = kTcConsumers / 32;

  if (tid == 0) {
    auto init = [](unsigned long long *b, int count) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count)
                   : "memory");
    };
    for (int s = 0; s < kTcRawStages; ++s) {
      init(&s_full[s], 1);
      init(&s_empty[s], kWarpsC);
    }
    for (int s = 0; s < kTcMaxStages; ++s) {
      init(&s_ready[s], kWarpsC);
      init(&s_freed[s], 1);
    }
    init(&s_accf, 1);
    init(&s_acce, kWarpsC);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
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
  // role timing: TMA lane (warp 0), MMA lane (warp 1), one slicing lane (warp 2)
  RoleClock rc((kTimed && lane == 0 && warp <= 2) ? A.phase : nullptr);
  RoleClock rtot((kTimed && tid == 0) ? A.phase : nullptr);

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      const uint32_t bytes = (uint32_t)(n * kTcKC * 4);
      uint32_t r = 0;
      bool ok = true;
      for (int64_t cell = blockIdx.x; cell < A.ncell && ok; cell += gridDim.x)
        for (int pass = A.rowmax ? 1 : 0; pass < 2 && ok; ++pass)
          for (int ch = 0; ch < nchunk; ++ch, ++r) {
            const int slot = (int)(r % kTcRawStages);
            rc.reset();
            if (r >= (uint32_t)kTcRawStages &&
                !bar_wait(smem_addr(&s_empty[slot]), ((r / kTcRawStages) - 1) & 1, &s_abort)) {
              ok = false;
              break;
            }
            rc.mark(16);
            tma_load(smem_addr(raw + (size_t)slot * kTcRawBytes), &xmap, ch * kTcKC,
                     (int)(cell * n), smem_addr(&s_full[slot]), bytes);
          }
      if (!ok) s_abort = 1;
      // every load issued has landed before the block gives up its shared memory
      for (uint32_t q = r > (uint32_t)kTcRawStages ? r - kTcRawStages : 0; q < r; ++q)
        bar_poll(smem_addr(&s_full[q % kTcRawStages]), (q / kTcRawStages) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t t = 0, cidx = 0;
      bool ok = true;
      for (int64_t cell = blockIdx.x; cell < A.ncell && ok; cell += gridDim.x, ++cidx) {
        // the previous cell's accumulators must have been read back
        rc.reset();
        if (cidx > 0 && !bar_wait(smem_addr(&s_acce), (cidx - 1) & 1, &s_abort)) {
          ok = false;
          break;
        }
        rc.mark(19);
        if (kTimed) atomicAdd(reinterpret_cast<unsigned long long *>(A.phase + 25), 1ull);
        for (int ch = 0; ch < nchunk; ++ch, ++t) {
          const uint32_t st = t % NS;
          rc.reset();
          if (!bar_wait(smem_addr(&s_ready[st]), (t / NS) & 1, &s_abort)) {
            ok = false;
            break;
          }
          rc.mark(17);
          fence_after();
          const uint32_t b0 = smem_addr(stages + (size_t)st * stage_bytes);
          for (int g = 0; g < P.ngroups; ++g) {
            const uint32_t idesc = umma_idesc(128, P.N[g]);
            const uint32_t da = b0 + (uint32_t)(P.a0[g] * sp) * kTcRowBytes;
            const uint32_t db = b0 + (uint32_t)(P.b0[g] * sp) * kTcRowBytes;
#pragma unroll
            for (int kk = 0; kk < kTcKC / 16; ++kk)
              mma_bf16(tmem + (uint32_t)P.col[g], umma_desc(da + kk * 32),
                       umma_desc(db + kk * 32), idesc, (ch > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(smem_addr(&s_freed[st]));
          if (ch + 1 == nchunk) mma_commit(smem_addr(&s_accf));
          rc.mark(18);
        }
      }
      if (!ok) s_abort = 1;
      // every committed MMA has completed before the tensor memory is given up
      if (t > 0) bar_poll(smem_addr(&s_freed[(t - 1) % NS]), ((t - 1) / NS) & 1);
    }
    __syncwarp();
  } else {
    const int ct = tid - 64;
    RoleClock &rcl = rc;
    const int items = n * (kTcKC / 4);  // (row, 4-column piece) per chunk
    constexpr int kItems = (64 * (kTcKC / 4) + kTcConsumers - 1) / kTcConsumers;
    uint32_t rc = 0, t = 0, cidx = 0;
    bool fail = false;
    for (int64_t cell = blockIdx.x; cell < A.ncell && !fail; cell += gridDim.x, ++cidx) {
      // row scales: from the given row maxima, else from a first pass over the chunks (the
      // 16 pieces of a row sit in 16 adjacent lanes)
      float mx[kItems];
#pragma unroll
      for (int q = 0; q < kItems; ++q) mx[q] = 0.f;
      bool ok = true;
      for (int ch = 0; !A.rowmax && ch < nchunk; ++ch, ++rc) {
        const int slot = (int)(rc % kTcRawStages);
        if (ok) ok = bar_wait(smem_addr(&s_full[slot]), (rc / kTcRawStages) & 1, &s_abort);
        if (ok) {
          const float *rs = reinterpret_cast<const float *>(raw + (size_t)slot * kTcRawBytes);
#pragma unroll
          for (int q = 0; q < kItems; ++q) {
            const int it = ct + q * kTcConsumers;
            if (it < items) {
              const float4 u = *reinterpret_cast<const float4 *>(rs + (it >> 4) * kTcKC + (it & 15) * 4);
              mx[q] = fmaxf(mx[q], fmaxf(fmaxf(fabsf(u.x), fabsf(u.y)), fmaxf(fabsf(u.z), fabsf(u.w))));
            }
          }
        }
        __syncwarp();
        if (lane == 0) bar_arrive(smem_addr(&s_empty[slot]));
      }
#pragma unroll
      for (int q = 0; q < kItems; ++q) {
        const int it = ct + q * kTcConsumers;
        if (A.rowmax) mx[q] = it < items ? A.rowmax[cell * A.rstride + (it >> 4)] : 0.f;
        for (int o = 1; o < 16; o <<= 1) mx[q] = fmaxf(mx[q], __shfl_xor_sync(0xffffffffu, mx[q], o));
        if (it < items && (it & 15) == 0) {
          int e = mx[q] > 0.f ? ilogbf(mx[q]) + 1 : 0;
          e = e < -100 ? -100 : (e > 100 ? 100 : e);
          rexp[it >> 4] = e;
          rinv[it >> 4] = ldexpf(1.0f, 6 - e);
        }
      }
      for (int i = ct; i < kTcLevels * ltri; i += kTcConsumers) Lacc[i] = 0;
      if (!consumers_and(ok)) {
        fail = true;
        break;
      }
      // slice each chunk into a free stage (row k*sp + a holds slice k of row a) and
      // hand it to the MMA issuer
      for (int ch = 0; ch < nchunk; ++ch, ++rc, ++t) {
        const int slot = (int)(rc % kTcRawStages);
        const uint32_t st = t % NS;
        if (warp == 2) rcl.mark(22);
        bool ok2 = bar_wait(smem_addr(&s_full[slot]), (rc / kTcRawStages) & 1, &s_abort);
        if (warp == 2) rcl.mark(20);
        // the MMAs that last read this stage must be complete
        if (ok2 && t >= NS) ok2 = bar_wait(smem_addr(&s_freed[st]), ((t / NS) - 1) & 1, &s_abort);
        if (warp == 2) rcl.mark(21);
        ok2 = __all_sync(0xffffffffu, ok2);  // the warp leaves together (it syncs below)
        if (!ok2) {
          s_abort = 1;
          ok = false;
          break;
        }
        unsigned char *buf = stages + (size_t)st * stage_bytes;
        const float *rs = reinterpret_cast<const float *>(raw + (size_t)slot * kTcRawBytes);
        for (int it = ct; it < items; it += kTcConsumers) {
          const int a = it >> 4, c4 = it & 15;
          const float4 u = *reinterpret_cast<const float4 *>(rs + a * kTcKC + c4 * 4);
          const float ra = rinv[a];
          uint64_t y01 = f2_mul(f2_pack(u.x, u.y), f2_pack(ra, ra));
          uint64_t y23 = f2_mul(f2_pack(u.z, u.w), f2_pack(ra, ra));
#pragma unroll
          for (int k = 0; k < kTcSlices; ++k) {
            // v_k = y rounded to a multiple of 2^-7k (round to nearest even by adding and
            // removing 1.5 * 2^(23 - 7k)); v_k 2^7k is an integer in [-64, 64]
            const uint64_t M = f2_pack(kSliceMagic[k], kSliceMagic[k]);
            const uint64_t v01 = f2_sub(f2_add(y01, M), M), v23 = f2_sub(f2_add(y23, M), M);
            if (k + 1 < kTcSlices) {
              y01 = f2_sub(y01, v01);
              y23 = f2_sub(y23, v23);
            }
            const int row = k * sp + a;
            uint2 w;
            w.x = pack2(__uint_as_float((uint32_t)v01), __uint_as_float((uint32_t)(v01 >> 32)));
            w.y = pack2(__uint_as_float((uint32_t)v23), __uint_as_float((uint32_t)(v23 >> 32)));
            *reinterpret_cast<uint2 *>(buf + (size_t)row * kTcRowBytes +
                                       ((((c4 >> 1) ^ (row & 7)) << 4) | ((c4 & 1) << 3))) = w;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          bar_arrive(smem_addr(&s_empty[slot]));
          bar_arrive(smem_addr(&s_ready[st]));
        }
      }
      // the cell's accumulators complete
      if (warp == 2) rcl.mark(22);
      if (ok) ok = bar_wait(smem_addr(&s_accf), cidx & 1, &s_abort);
      if (warp == 2) rcl.mark(24);
      if (!consumers_and(ok)) {
        fail = true;
        break;
      }
      fence_after();
      // read the accumulators back.  The three warps of a lane quarter share each
      // group's 8-column blocks round robin, four loads in flight before one wait.  The
      // accumulator of slice product (k, l) holds 2^-7(k+l) D with D = S_k S_l^T an
      // integer matrix; every owned D_ij is added, as the exact integer it is, to the
      // level k + l accumulator of entry (min(i,j), max(i,j)) (for k != l, D_ij and D_ji
      // both belong to C_ij, so D_ii counts twice; for k == l, D is symmetric and only
      // i <= j is taken).  Integer addition makes the order irrelevant.
      {
        const int q4 = warp & 3, sub = (warp - 2) >> 2;  // lanes 32 q4 .. 32 q4 + 31
        const int lrow = 32 * q4 + lane;                  // accumulator lane = row of A
        const int na = 128 / sp;
        for (int g = 0; g < P.ngroups; ++g) {
          const int il = lrow / sp, i = lrow - il * sp, k = P.a0[g] + il;
          const bool row_ok = il < na && i < n && k < kTcSlices;
          uint32_t ownl = 0;  // B slices l whose product (k, l) this group owns
          if (row_ok)
            for (int l = 0; l < kTcSlices; ++l)
              if (P.own[k * kTcSlices + l] == g + 1) ownl |= 1u << l;
          const int nblk = P.N[g] / 8;
          for (int b0 = sub; b0 < nblk; b0 += 4 * 3) {
            uint32_t r[4][8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int b = b0 + 3 * q;
              if (b < nblk)  // warp-uniform
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]), "=r"(r[q][4]),
                      "=r"(r[q][5]), "=r"(r[q][6]), "=r"(r[q][7])
                    : "r"(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(P.col[g] + 8 * b))
                    : "memory");
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int b = b0 + 3 * q;
              if (b >= nblk) continue;
              const int jl = (8 * b) / sp, j0 = 8 * b - jl * sp, l = P.b0[g] + jl;
              if (!row_ok || jl >= P.nb[g] || !((ownl >> l) & 1u)) continue;
              const float scale = kLevelScale[k + l];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int j = j0 + u;
                if (j >= n || (k == l && i > j)) continue;
                const int tri = i <= j ? tri_row(n, i) + (j - i) : tri_row(n, j) + (i - j);
                const int d = __float2int_rn(__uint_as_float(r[q][u]) * scale);
                // a diagonal entry of a k != l product is its own transpose: counted twice
                atomicAdd(&Lacc[(k + l) * ltri + tri], (k != l && i == j) ? 2 * d : d);
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(smem_addr(&s_acce));  // the accumulators may be reused
      consumers_sync();
      // C_ab = 2^(e_a + e_b - 12) sum_m 2^(-7 m) L_m, formed exactly in integers:
      // T = sum_{m <= 4} L_m 2^(28 - 7m) and U = sum_{m >= 5} L_m 2^(49 - 7m) (|L_m| < 2^28,
      // so |T| < 2^60), C_ab = 2^(e_a + e_b - 40) (T + 2^-21 U); written once rounded, as a
      // double-float pair or a double
      for (int e = ct; e < ntri; e += kTcConsumers) {
        int a = 0;  // entry e of the upper triangle, row by row: (a, b)
        while (a + 1 < n && tri_row(n, a + 1) <= e) ++a;
        const int b = a + (e - tri_row(n, a)), w = e;
        long long T = 0, U = 0;
#pragma unroll
        for (int m = 0; m <= 4; ++m) T = T * 128 + Lacc[m * ltri + w];
#pragma unroll
        for (int m = 5; m < kTcLevels; ++m) U = U * 128 + Lacc[m * ltri + w];
        const int sc = rexp[a] + rexp[b] - 40;
        if (A.Cd) {
          const double v = ldexp((double)T, sc) + ldexp((double)U, sc - 21);
          double *C = A.Cd + cell * A.cstride;
          C[a * n + b] = v;
          C[b * n + a] = v;
        } else {
          const float th = __ll2float_rn(T);
          const long long tr = T - __float2ll_rn(th);  // exact: th is an integer
          const float tl = __fadd_rn(__ll2float_rn(tr), ldexpf(__ll2float_rn(U), -21));
          const float hi = __fadd_rn(th, tl);
          const float lo = __fsub_rn(tl, __fsub_rn(hi, th));
          float2 *C = A.C + cell * A.cstride;
          const float2 v = make_float2(ldexpf(hi, sc), ldexpf(lo, sc));
          C[a * n + b] = v;
          C[b * n + a] = v;
        }
      }
      if (ct == 0 && A.disc) A.disc[cell] = 0.0;
      consumers_sync();  // the level accumulators are free for the next cell
      if (warp == 2) rcl.mark(23);
    }
    if (fail && ct == 0) {
      s_abort = 1;
      atomicOr(A.flag, 2);
    }
  }
  rtot.mark(26);
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

// cuTensorMapEncodeTiled through the driver's entry point (no link against the
// driver library); null if unavailable
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static bool looked_up = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!looked_up) {
    looked_up = true;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", reinterpret_cast<void **>(&fn),
                                         12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      fn = nullptr;
    }
  }
  return fn;
}
}  // namespace

int gram_tc_prepare(int n) {
  const GramTcPlan p = gram_tc_plan(n);
  if (p.ngroups == 0 || !encode_tiled()) return -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  const size_t smem = launch_smem(p);
  if (smem <= g_opted) return 0;
  if (cudaFuncSetAttribute(gram_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(gram_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
                   double *Cd, int64_t cstride, double *disc, int *flag, cudaStream_t s,
                   const float *rowmax, int64_t rstride, long long *phase) {
  if (ncell <= 0) return 0;
  // the cells' rows must form one row-major [ncell * n][K] array for the tensor map
  if (!gram_tc_supported(n, K) || xstride != (int64_t)n * K ||
      (reinterpret_cast<uintptr_t>(X) & 15) != 0 || ncell * n > 0x7fffffffLL)
    return -1;
  TcArgs a{};
  a.ncell = ncell;
  a.K = K;
  a.C = C;
  a.Cd = Cd;
  a.cstride = cstride;
  a.disc = disc;
  a.flag = flag;
  a.rowmax = rowmax;
  a.rstride = rstride;
  a.phase = phase;
  a.plan = gram_tc_plan(n);
  const size_t smem = launch_smem(a.plan);
  if (smem > g_opted) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap != cudaStreamCaptureStatusNone || gram_tc_prepare(n) != 0) return -1;
  }
  const EncodeTiled enc = encode_tiled();
  if (!enc) return -1;
  // X as a 2-D FP32 array [ncell * n][K] (K innermost), boxes of n rows x 64 columns;
  // columns beyond K (a ragged last chunk) read as zeros
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)(ncell * n)};
  const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcKC, (cuuint32_t)n};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return -1;
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(ncell < sms ? ncell : sms);
  if (phase)
    gram_tc_kernel<true><<<grid, kTcThreadsAll, smem, s>>>(map, a);
  else
    gram_tc_kernel<false><<<grid, kTcThreadsAll, smem, s>>>(map, a);
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
