// FP64 products on the 16-bit tensor cores (tcgen05), exact to FP64 level, operands fed by TMA.
//
// GB300 retires 2 FP64 FMAs per SM per clock but thousands of 16-bit tensor-core FMAs, and the
// method's large products -- the ARA samples Y = T Omega and projections B = T^T Q of the generated
// tiles (Algorithm 1 on Section 6's kernel tiles), the sampling chains of Equation 2 with the
// factor's U and V panels, batchTrsm -- are dense contractions.  They are computed by error-free
// splitting (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012):
//
//  * Every entry x of an operand is written as x = 2^e * sum_{i=1..8} x_i 2^(-7 i) with integers
//    |x_i| <= 127, where 2^e bounds the operand block (the whole tile for T, each column for Omega
//    and Q).  The x_i are the 7-bit chunks of the 56-bit truncation of |x| 2^(56-e) with the sign of
//    x, found with integer operations on the FP64 bit pattern and stored as int8: 8 bytes per
//    entry, the bytes of the FP64 operand.  Truncation error < 2^(e-56).
//  * The product keeps the chunk pairs (i, j) with i + j <= S + 1 (S = 8: every pair of weight
//    >= 2^-63 of the block bounds; S < 8 truncates both operands to 7S bits, the precision knob of
//    the mixed path).  Chunks are exact in FP16 (and BF16); a chunk product is below 2^14
//    and the sum of one group g = i + j - 2 over 128 consecutive k, added over its g + 1 pairs, stays
//    below 2^24: the FP32 accumulation of the tensor core is exact.  Every 128 k the group sums move
//    from tensor memory to 32-bit integer totals (exact for K <= 16384), combined once at the end.
//
// Kernel structure (one CTA = 128 output rows x 16 output columns x one K slice, 320 threads):
//  * warp 0: TMA producer.  Boxes of the int8 chunk planes of A and B (one per plane) are copied by
//    cp.async.bulk.tensor into a 2-stage ring (32 k per stage), mbarrier completion.  Operands
//    stored along k are read through a 4D view (16 k, rows, k / 16, plane), so a stage holds each
//    16-k half as [row][16 bytes] and a warp's 16-byte reads of consecutive rows are contiguous.
//  * warps 2-5: converters.  Thread t owns row t of the A tile (and one stacked row of B): int8 chunks
//    become FP16 (two byte permutes and one f16x2 subtraction per pair) in the canonical K-major
//    layout of the tensor core (8-row x 16-byte core matrices; either orientation of A in HBM lands
//    in the same layout), into one of four chunk buffers, so conversion runs ahead of the MMAs.
//  * warp 1: one thread issues tcgen05.mma (kind::f16, FP16 in, FP32 accumulate in tensor memory).
//    For a 16-k step and A slice i, B is the stack [B_1 | ... | B_(S+1-i)] (N = 16 (S + 1 - i)) and
//    the accumulator starts at the column block of group i - 1: every group sum accumulates in place.
//    Two 128-column accumulator buffers alternate between 128-k windows.
//  * warps 6-9: epilogue.  They drain each window's group sums (tcgen05.ld) into integer totals
//    while the next window accumulates, then recombine in FP64 and store (or write split-K partials,
//    summed in slice order by the last CTA of each output block).
// Every wait is bounded: on a timeout the CTA sets a device flag, lets its copies land, frees its
// tensor memory and returns; the host reports TLR_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "common.h"

namespace tlr {

__device__ int g_oz_timeout = 0;
// statistics: CTAs by planes used ([s], s = 1..8) and chunk bytes of the operands read ([9]: each
// A block counted once per output-column block 0, each B block once per row block 0)
__device__ unsigned long long g_oz_stats[10];

namespace {

constexpr int OZ_S = 8;       // chunk planes per operand
constexpr int OZ_TM = 128;    // output rows per CTA (tcgen05 M)
constexpr int OZ_TN = 16;     // output columns per CTA
constexpr int OZ_KS = 32;     // k per TMA stage
constexpr int OZ_KC = 16;     // k per MMA
constexpr int OZ_CW = 8;      // 16-k steps per exact window (128 k)
constexpr int OZ_NST = 4;     // int8 stages in flight
constexpr int OZ_NBF = 4;     // FP16 chunk buffers between the converters and the MMA issuer
constexpr int OZ_THREADS = 320;
constexpr int ST_A = OZ_S * OZ_TM * OZ_KS;        // int8 A per stage (32 KB)
constexpr int ST_B = OZ_S * OZ_TN * OZ_KS;        // int8 B per stage (4 KB)
constexpr int ST_BYTES = ST_A + ST_B;
constexpr int BF_B = OZ_S * OZ_TN * OZ_KC * 2;    // stacked FP16 B chunk in shared memory, 128 rows (4 KB)
constexpr int BF_BYTES = BF_B;
// Tensor memory: two accumulator buffers of 8 groups x 16 columns (columns 0-255), then OZ_NBF FP16
// A chunks (128 lanes = rows; 8 planes x 8 columns, each column two k values)
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_TMEM_A = 256;
constexpr int OZ_A_COLS = OZ_S * OZ_KC / 2;       // 64 columns per A chunk
constexpr int OZ_SMEM = 1024 + OZ_NST * ST_BYTES + OZ_NBF * BF_BYTES + 256;
static_assert(OZ_TMEM_A + OZ_NBF * OZ_A_COLS <= OZ_TMEM_COLS, "tensor memory budget");
constexpr unsigned long long OZ_WAIT_NS = 2000000000ull;

// Tensor maps live in the job table (global memory); CUtensorMap carries its own (>= 64-byte)
// alignment, and the upload ring hands out 256-byte aligned regions.
struct OzDev {
  CUtensorMap ta, tb, ta0;  // ta0: the first K segment of A (K0 > 0)
  const int* eA;
  const int* eB;
  double* C;
  double* ws;
  int* ctr;
  double tol;  // > 0: truncate to the fewest planes whose error bound per entry stays below tol
  int M, N, K, ldc, acol, accumulate, eB_stride, nsplit, tiles_n, S, smin, K0;
};
static_assert(alignof(OzDev) >= 64 && sizeof(OzDev) % 64 == 0, "tensor maps need 64-byte alignment");

inline int64_t oz_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Exponent e with |x| < 2^e for the largest |x| recorded as FP64 bits (0 for an all-zero block).
__device__ __forceinline__ int oz_exponent(unsigned long long maxbits) {
  const int ex = (int)((maxbits >> 52) & 0x7FF);
  return ex == 0 ? 0 : ex - 1022;
}

// The eight signed 7-bit chunks of x relative to 2^e.
__device__ __forceinline__ void oz_split(double x, int e, int8_t out[OZ_S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long F = 0;
  if (ex != 0) {  // subnormals are below every block bound used here: they truncate to zero
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int shift = ex - e - 1019;  // F = floor(|x| 2^(56 - e)) < 2^56
    if (shift >= 0) F = mant << shift;
    else if (shift > -64) F = mant >> (-shift);
  }
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const int c = (int)((F >> (49 - 7 * i)) & 127);
    out[i] = (int8_t)(neg ? -c : c);
  }
}

// ---- PTX wrappers (tcgen05, TMA, mbarrier)
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// try_wait with a suspend-time hint: a waiting thread sleeps until the phase completes (or 20 us
// pass) instead of taking issue slots from the converter warps.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p;}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(20000)
      : "memory");
  return ok != 0;
}
// Bounded wait on a barrier phase; a timeout (or another role's abort) returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    if (gtimer() - t0 > OZ_WAIT_NS) {
      *abort = 1;
      atomicExch(&g_oz_timeout, 1);
      return false;
    }
  }
}
// Bounded wait that ignores aborts (for copies and MMAs that must land before the CTA exits).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > OZ_WAIT_NS) {
      atomicExch(&g_oz_timeout, 1);
      return;
    }
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                       uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor, K-major, no swizzle: lbo = byte stride between core matrices
// along K, sbo = byte stride between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major, M x N.
__device__ __forceinline__ uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
  asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}" ::"r"(
                   dtmem),
               "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
               : "memory");
}
// The same with the A operand in tensor memory (lane = row, each 32-bit column two consecutive k).
__device__ __forceinline__ void umma_f16_ts(uint32_t dtmem, uint32_t atmem, uint64_t bd, uint32_t idesc, int acc) {
  asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;}" ::"r"(
                   dtmem),
               "r"(atmem), "l"(bd), "r"(idesc), "r"(acc)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Four signed int8 chunks (one word) -> two packed FP16 pairs: with u = c + 128 (the byte XOR
// 0x80), the FP16 bit pattern 0x6400 + u is 1024 + u, and subtracting 1152 leaves c exactly.
__device__ __forceinline__ uint32_t oz_hsub(uint32_t h) {
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(0x64806480u));
  return r;
}
__device__ __forceinline__ void oz_cvt4(uint32_t w, uint32_t& lo, uint32_t& hi) {
  const uint32_t u = w ^ 0x80808080u;
  lo = oz_hsub(__byte_perm(u, 0x64646464u, 0x5140u));
  hi = oz_hsub(__byte_perm(u, 0x64646464u, 0x7362u));
}
// 16 int8 chunks (4 words) -> 16 FP16 (8 words)
__device__ __forceinline__ void oz_cvt16(const uint32_t (&w)[4], uint32_t (&o)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) oz_cvt4(w[q], o[2 * q], o[2 * q + 1]);
}

// Drain accumulator window w (buffer w & 1) of this thread's TMEM lane into the integer totals (each
// group of a window is an integer below 2^24; over K <= 16384 a total stays below 2^31) and release
// the buffer to the MMA issuer.
__device__ __forceinline__ bool oz_drain(int w, int S, uint32_t b_accf, uint32_t b_acce, uint32_t tmem, int lq,
                                         volatile int* abort, int (&tot)[OZ_S][OZ_TN]) {
  const int buf = w & 1;
  if (!mbar_wait(b_accf + 8 * buf, (w >> 1) & 1, abort)) return false;
  tc_fence_after();
  const uint32_t ta = tmem + ((uint32_t)(32 * lq) << 16) + buf * 128;
#pragma unroll
  for (int g = 0; g < OZ_S; ++g)
    if (g < S) {
      uint32_t r[16];
      tmem_ld16(ta + OZ_TN * g, r);
#pragma unroll
      for (int c = 0; c < OZ_TN; ++c) tot[g][c] += __float2int_rn(__uint_as_float(r[c]));
    }
  tc_fence_before();
  mbar_arrive(b_acce + 8 * buf);
  return true;
}

}  // namespace

// ------------------------------------------------------------------ splitting
// Chunks of a batch of dense tiles (n x n each, column-major) relative to each tile's bound,
// written twice: Sc (same layout as T: row k of T^T is contiguous) and Sr (transposed: row m of T
// contiguous), so that both T Omega and T^T Q read their left operand along k.
// CTA = one 32 x 32 block of one tile; the transposed copy goes through shared memory.
__global__ void __launch_bounds__(256) k_oz_split_tiles(const double* __restrict__ T, int n,
                                                        const unsigned long long* __restrict__ tmax,
                                                        int8_t* __restrict__ Sc, int8_t* __restrict__ Sr,
                                                        int* __restrict__ eT) {
  const int t = blockIdx.z;
  const int e = oz_exponent(tmax[t]);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) eT[t] = e;
  const size_t n2 = (size_t)n * n;
  const double* x = T + (size_t)t * n2;
  int8_t* oc = Sc ? Sc + (size_t)t * OZ_S * n2 : nullptr;
  int8_t* orow = Sr + (size_t)t * OZ_S * n2;
  __shared__ int8_t tr[OZ_S][32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int kk = ty; kk < 32; kk += 8) {
    const int m = m0 + tx, k = k0 + kk;
    int8_t sl[OZ_S];
    if (m < n && k < n) oz_split(x[m + (size_t)k * n], e, sl);
    else
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) sl[q] = 0;
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) {
      if (oc && m < n && k < n) oc[(size_t)q * n2 + m + (size_t)k * n] = sl[q];
      tr[q][kk][tx] = sl[q];
    }
  }
  __syncthreads();
  for (int mm = ty; mm < 32; mm += 8) {
    const int m = m0 + mm, k = k0 + tx;
    if (m < n && k < n)
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) orow[(size_t)q * n2 + k + (size_t)m * n] = tr[q][tx][mm];
  }
}

// Chunks of column blocks X_j (K x ncols_j, leading dimension ld_j) relative to each column's
// bound; plane q of column c of block j lands at Xs_j + q * plane + c * ldo (rows K .. ldo-1 zero).
// One CTA per column.
__global__ void __launch_bounds__(256) k_oz_split_cols(const OzColJob* __restrict__ jobs,
                                                       const int* __restrict__ col_job) {
  const int g = blockIdx.x;
  const OzColJob J = jobs[col_job[g]];
  const int K = J.K;
  const int c = g - J.col0;
  const double* x = J.X + (size_t)c * J.ld;
  const int ldo = J.tld > 0 ? K : (J.ldo > 0 ? J.ldo : oz_ld(K));
  const size_t plane = J.plane > 0 ? J.plane : (size_t)J.ncols * ldo;
  const size_t kst = J.tld > 0 ? (size_t)J.tld : 1;  // stride of k in the output
  int8_t* xs = J.tld > 0 ? J.Xs + c : J.Xs + (size_t)c * ldo;
  int e;
  if (J.efix != OZ_EFIX_NONE || J.emax) {
    e = J.emax ? oz_exponent(*J.emax) : J.efix;
    if (J.emax && J.e && c == 0 && threadIdx.x == 0) J.e[0] = e;
  } else {
    __shared__ unsigned long long red[8];
    unsigned long long m = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(x[k]));
      m = b > m ? b : m;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
      m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
      red[0] = m;
    }
    __syncthreads();
    e = oz_exponent(red[0]);
    if (threadIdx.x == 0) J.e[c] = e;
  }
  for (int k = threadIdx.x; k < ldo; k += blockDim.x) {
    int8_t s[OZ_S];
    if (k < K) oz_split(x[k], e, s);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) xs[(size_t)q * plane + k * kst] = k < K ? s[q] : (int8_t)0;
  }
}

// ------------------------------------------------------------------ product
// C(M x N) = 2^(eA + eB_n) * sum over chunk pairs (i, j), i + j <= S + 1, of A_i B_j 2^(-7(i+j)),
// A(m, k) = A_i[k + m lda] (rows along k) or, with acol, A_i[m + k lda]; B(k, n) = B_j[k + n ldb].
// Grid (ceil(M / 128), tiles_n * nsplit, jobs).
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_mma(const OzDev* __restrict__ jobs) {
  const OzDev* Jp = jobs + blockIdx.z;
  const int tiles_n = Jp->tiles_n, nsplit = Jp->nsplit;
  if ((int)blockIdx.y >= tiles_n * nsplit) return;
  const int nt = blockIdx.y % tiles_n, split = blockIdx.y / tiles_n;
  const int M = Jp->M, N = Jp->N, K = Jp->K, acol = Jp->acol;
  const int m0 = blockIdx.x * OZ_TM, n0 = nt * OZ_TN;
  if (m0 >= M || n0 >= N) return;
  // Planes used: S, or with a tolerance the fewest s >= smin whose bound K (s + 1) 2^(eA + eB - 7 s)
  // on every entry's error (truncation of both operands to 7s bits plus the dropped chunk pairs;
  // eB = the largest column exponent of this CTA) is below tol.  Uniform over the CTA.
  int S = Jp->S;
  if (Jp->tol > 0.0) {
    int eb = -100000;
    for (int c = 0; c < OZ_TN; ++c)
      if (n0 + c < N) eb = max(eb, Jp->eB[(n0 + c) * Jp->eB_stride]);
    const int ea = *Jp->eA;
    for (int s = Jp->smin; s < S; ++s)
      if (ldexp((double)K * (s + 1), ea + eb - 7 * s) <= Jp->tol) {
        S = s;
        break;
      }
  }
  const int nst_all = (K + OZ_KS - 1) / OZ_KS;
  const int sb = (int)((int64_t)nst_all * split / nsplit), se = (int)((int64_t)nst_all * (split + 1) / nsplit);
  const int nst = se - sb;            // TMA stages of this K slice
  if (threadIdx.x == 0) {
    const int kl = min(se * OZ_KS, K) - sb * OZ_KS;
    unsigned long long by = 0;
    if (nt == 0) by += (unsigned long long)S * min(OZ_TM, M - m0) * kl;
    if (blockIdx.x == 0) by += (unsigned long long)S * min(OZ_TN, N - n0) * kl;
    atomicAdd(&g_oz_stats[S], 1ull);
    atomicAdd(&g_oz_stats[9], by);
  }
  const int nch = 2 * nst;            // 16-k MMA steps
  const int nwin = (nch + OZ_CW - 1) / OZ_CW;

  extern __shared__ uint8_t oz_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = base;                           // OZ_NST stages of int8 A then B
  uint8_t* bfb = ring + OZ_NST * ST_BYTES;        // OZ_NBF FP16 chunk buffers: A planes then stacked B
  uint64_t* bars = reinterpret_cast<uint64_t*>(bfb + OZ_NBF * BF_BYTES);
  // barriers: full8[OZ_NST] empty8[OZ_NST] fullbf[OZ_NBF] emptybf[OZ_NBF] accf[2] acce[2] fin
  const uint32_t b_full8 = su32(bars), b_empty8 = su32(bars + OZ_NST), b_fullbf = su32(bars + 2 * OZ_NST),
                 b_emptybf = su32(bars + 2 * OZ_NST + OZ_NBF), b_accf = su32(bars + 2 * OZ_NST + 2 * OZ_NBF),
                 b_acce = b_accf + 16, b_fin = b_accf + 32;
  volatile int* abort = reinterpret_cast<volatile int*>(bars + 2 * OZ_NST + 2 * OZ_NBF + 5);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_NST + 2 * OZ_NBF + 6);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < OZ_NST; ++s) {
      mbar_init(b_full8 + 8 * s, 1);
      mbar_init(b_empty8 + 8 * s, 128);
    }
    for (int s = 0; s < OZ_NBF; ++s) {
      mbar_init(b_fullbf + 8 * s, 128);
      mbar_init(b_emptybf + 8 * s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(b_accf + 8 * s, 1);
      mbar_init(b_acce + 8 * s, 128);
    }
    mbar_init(b_fin, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&Jp->ta) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&Jp->tb) : "memory");
      const int K0 = Jp->K0;
      if (K0 > 0) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&Jp->ta0) : "memory");
      const uint32_t bytes = (uint32_t)(S * (OZ_TM * OZ_KS + OZ_TN * OZ_KS));  // one box per plane
      int issued = 0;
      for (int s = 0; s < nst; ++s) {
        const int slot = s % OZ_NST;
        if (!mbar_wait(b_empty8 + 8 * slot, ((s / OZ_NST) & 1) ^ 1, abort)) break;
        uint8_t* st = ring + slot * ST_BYTES;
        const int k0 = (sb + s) * OZ_KS;
        mbar_expect_tx(b_full8 + 8 * slot, bytes);
        for (int q = 0; q < S; ++q) {
          if (acol) tma_3d(su32(st + q * (OZ_TM * OZ_KS)), &Jp->ta, m0, k0, q, b_full8 + 8 * slot);
          else if (k0 < K0) tma_4d(su32(st + q * (OZ_TM * OZ_KS)), &Jp->ta0, 0, m0, k0 / 16, q, b_full8 + 8 * slot);
          else tma_4d(su32(st + q * (OZ_TM * OZ_KS)), &Jp->ta, 0, m0, (k0 - K0) / 16, q, b_full8 + 8 * slot);
          tma_4d(su32(st + ST_A + q * (OZ_TN * OZ_KS)), &Jp->tb, 0, n0, k0 / 16, q, b_full8 + 8 * slot);
        }
        issued = s + 1;
      }
      // every issued copy lands before the CTA can exit
      for (int s = issued > OZ_NST ? issued - OZ_NST : 0; s < issued; ++s)
        mbar_drain(b_full8 + 8 * (s % OZ_NST), (s / OZ_NST) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t bf0 = su32(bfb);
      for (int c = 0; c < nch; ++c) {
        const int sbf = c % OZ_NBF;
        if (!mbar_wait(b_fullbf + 8 * sbf, (c / OZ_NBF) & 1, abort)) break;
        const int w = c / OZ_CW, buf = w & 1;
        const bool first = (c % OZ_CW) == 0;
        if (first && !mbar_wait(b_acce + 8 * buf, ((w >> 1) & 1) ^ 1, abort)) break;
        tc_fence_after();
        const uint64_t bd = umma_desc(bf0 + sbf * BF_BYTES, OZ_S * OZ_TN * 16, 128);
        const uint32_t at = tmem + OZ_TMEM_A + sbf * OZ_A_COLS;
#pragma unroll 1
        for (int i = 0; i < S; ++i)
          umma_f16_ts(tmem + buf * 128 + OZ_TN * i, at + i * (OZ_KC / 2), bd, umma_idesc(OZ_TM, OZ_TN * (S - i)),
                      (first && i == 0) ? 0 : 1);
        umma_commit(b_emptybf + 8 * sbf);
        if ((c % OZ_CW) == OZ_CW - 1 || c == nch - 1) umma_commit(b_accf + 8 * buf);
      }
      umma_commit(b_fin);  // arrives when every MMA of this thread has completed
      mbar_drain(b_fin, 0);
    }
  } else if (warp < 6) {
    // ---------------- converters (warps 2-5): int8 chunks -> FP16.  A warp may reach only its quarter
    // of the tensor-memory lanes, so thread (warp, lane) owns A row 32 (warp % 4) + lane, written to
    // the chunk's A buffer in tensor memory (one 8-column store per plane); thread t = tid - 64 owns
    // stacked B row t when t < 16 S, written to shared memory in the canonical K-major layout.
    const int t = tid - 64;
    const int row = 32 * (warp & 3) + lane;
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + OZ_TMEM_A;
    bool ok = true;
    for (int s = 0; s < nst && ok; ++s) {
      const int slot = s % OZ_NST;
      if (!mbar_wait(b_full8 + 8 * slot, (s / OZ_NST) & 1, abort)) break;
      const uint8_t* a8 = ring + slot * ST_BYTES;
      const uint8_t* b8 = a8 + ST_A;
      for (int h = 0; h < 2; ++h) {
        const int c = 2 * s + h, sbf = c % OZ_NBF;
        if (!mbar_wait(b_emptybf + 8 * sbf, ((c / OZ_NBF) & 1) ^ 1, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint8_t* bbf = bfb + sbf * BF_BYTES;
        uint32_t w[OZ_S][4];
        if (acol) {  // stage image [q][k 32][m 128]: 16 byte loads per plane
#pragma unroll
          for (int q = 0; q < OZ_S; ++q)
            if (q < S) {
              const uint8_t* p = a8 + q * (OZ_TM * OZ_KS) + (16 * h) * OZ_TM + row;
#pragma unroll
              for (int u = 0; u < 4; ++u)
                w[q][u] = __byte_perm(
                    __byte_perm((uint32_t)p[(4 * u) * OZ_TM], (uint32_t)p[(4 * u + 1) * OZ_TM], 0x0040u),
                    __byte_perm((uint32_t)p[(4 * u + 2) * OZ_TM], (uint32_t)p[(4 * u + 3) * OZ_TM], 0x0040u), 0x5410u);
            }
        } else {  // stage image [q][half 2][m 128][16 k]: one contiguous 16-byte load per plane
#pragma unroll
          for (int q = 0; q < OZ_S; ++q)
            if (q < S) {
              const uint4 v = *reinterpret_cast<const uint4*>(a8 + q * (OZ_TM * OZ_KS) + h * (OZ_TM * 16) + row * 16);
              w[q][0] = v.x;
              w[q][1] = v.y;
              w[q][2] = v.z;
              w[q][3] = v.w;
            }
        }
        const uint32_t ta = trow + sbf * OZ_A_COLS;
#pragma unroll
        for (int q = 0; q < OZ_S; ++q)
          if (q < S) {
            uint32_t o[8];
            oz_cvt16(w[q], o);
            tmem_st8(ta + q * (OZ_KC / 2), o);
          }
        if (t < OZ_TN * S) {  // B image [q][half 2][n 16][16 k] -> stacked row t
          const uint4 v = *reinterpret_cast<const uint4*>(b8 + (t / OZ_TN) * (OZ_TN * OZ_KS) + h * (OZ_TN * 16) +
                                                          (t % OZ_TN) * 16);
          const uint32_t wb[4] = {v.x, v.y, v.z, v.w};
          uint32_t o[8];
          oz_cvt16(wb, o);
          uint8_t* d = bbf + t * 16;
          *reinterpret_cast<uint4*>(d) = make_uint4(o[0], o[1], o[2], o[3]);
          *reinterpret_cast<uint4*>(d + OZ_S * OZ_TN * 16) = make_uint4(o[4], o[5], o[6], o[7]);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        mbar_arrive(b_fullbf + 8 * sbf);
      }
      mbar_arrive(b_empty8 + 8 * slot);
    }
  } else {
    // ---------------- epilogue (warps 6-9): window drains, FP64 recombination, store
    const int lq = warp & 3, row = 32 * lq + lane, m = m0 + row;
    int tot[OZ_S][OZ_TN];
#pragma unroll
    for (int g = 0; g < OZ_S; ++g)
#pragma unroll
      for (int c = 0; c < OZ_TN; ++c) tot[g][c] = 0;
    bool ok = true;
    for (int w = 0; w < nwin && ok; ++w) ok = oz_drain(w, S, b_accf, b_acce, tmem, lq, abort, tot);
    // group g has weight 2^-7(g+2): hi = groups 0-3 and lo = groups 4-7, both below 2^53 (exact in
    // 64-bit integers and in FP64); value = (hi 2^28 + lo) 2^-63 (one rounding)
    long long hi[OZ_TN], lo[OZ_TN];
#pragma unroll
    for (int c = 0; c < OZ_TN; ++c) {
      hi[c] = ((long long)tot[0][c] << 21) + ((long long)tot[1][c] << 14) + ((long long)tot[2][c] << 7) + tot[3][c];
      lo[c] = ((long long)tot[4][c] << 21) + ((long long)tot[5][c] << 14) + ((long long)tot[6][c] << 7) + tot[7][c];
    }
    const int eA = *Jp->eA;
    double* Cp = Jp->C;
    const int ldc = Jp->ldc;
    const size_t MN = (size_t)M * N;
#pragma unroll
    for (int c = 0; c < OZ_TN; ++c) {
      const int n = n0 + c;
      if (m < M && n < N) {
        double v = fma((double)hi[c], 268435456.0, (double)lo[c]);
        v = ldexp(v, eA + Jp->eB[n * Jp->eB_stride] - 63);
        if (nsplit > 1) {
          Jp->ws[(size_t)split * MN + m + (size_t)n * M] = v;
        } else {
          double* cp = Cp + m + (size_t)n * ldc;
          *cp = Jp->accumulate ? *cp + v : v;
        }
      }
    }
    if (nsplit > 1) {
      // the last slice to finish this output block sums the partials in slice order
      __threadfence();
      asm volatile("bar.sync 1, 128;" ::: "memory");
      __shared__ int last;
      int* ctr = Jp->ctr + (m0 / OZ_TM) * tiles_n + nt;
      if (row == 0) last = (atomicAdd(ctr, 1) == nsplit - 1);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (last) {
        __threadfence();
        if (m < M)
          for (int c = 0; c < OZ_TN; ++c) {
            const int n = n0 + c;
            if (n >= N) break;
            const size_t o = m + (size_t)n * M;
            double v = 0.0;
            for (int sp = 0; sp < nsplit; ++sp) v += __ldcg(Jp->ws + (size_t)sp * MN + o);
            double* cp = Cp + m + (size_t)n * ldc;
            *cp = Jp->accumulate ? *cp + v : v;
          }
        if (row == 0) *ctr = 0;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
  }
}

// Largest |entry| of each of a batch of n2-element blocks, as FP64 bits (atomic max; zeroed first).
__global__ void k_oz_absmax(const double* __restrict__ T, int64_t n2, unsigned long long* __restrict__ tmax) {
  const double* x = T + (size_t)blockIdx.y * n2;
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(tmax + blockIdx.y, (unsigned long long)__double_as_longlong(m));
}

void oz_absmax(tlr_ctx* ctx, int nblocks, int64_t n2, const double* T, unsigned long long* tmax) {
  if (nblocks <= 0) return;
  TLR_CUDA(cudaMemsetAsync(tmax, 0, sizeof(unsigned long long) * nblocks, ctx->stream));
  dim3 grid((unsigned)std::min<int64_t>(oz_cdiv(n2, 256), 64), (unsigned)nblocks);
  TLR_SITE_PRE(ctx);
  k_oz_absmax<<<grid, 256, 0, ctx->stream>>>(T, n2, tmax);
  TLR_LAUNCH_CHECK(ctx);
}

void oz_split_tiles(tlr_ctx* ctx, int ntiles, int n, const double* T, const unsigned long long* tmax, int8_t* Sc,
                    int8_t* Sr, int* eT) {
  if (ntiles <= 0) return;
  dim3 grid((unsigned)oz_cdiv(n, 32), (unsigned)oz_cdiv(n, 32), (unsigned)ntiles);
  TLR_SITE_PRE(ctx);
  k_oz_split_tiles<<<grid, 256, 0, ctx->stream>>>(T, n, tmax, Sc, Sr, eT);
  TLR_LAUNCH_CHECK(ctx);
}

void oz_split_cols(tlr_ctx* ctx, std::vector<OzColJob>& jobs) {
  std::vector<int> col_job;
  for (size_t j = 0; j < jobs.size(); ++j) {
    jobs[j].col0 = (int)col_job.size();
    for (int c = 0; c < jobs[j].ncols; ++c) col_job.push_back((int)j);
  }
  if (col_job.empty()) return;
  const OzColJob* dj = static_cast<const OzColJob*>(upload(ctx, jobs.data(), jobs.size() * sizeof(OzColJob)));
  const int* dc = static_cast<const int*>(upload(ctx, col_job.data(), col_job.size() * sizeof(int)));
  TLR_SITE_PRE(ctx);
  k_oz_split_cols<<<(unsigned)col_job.size(), 256, 0, ctx->stream>>>(dj, dc);
  TLR_LAUNCH_CHECK(ctx);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  TLR_REQUIRE(fn != nullptr, TLR_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  return fn;
}

void encode(CUtensorMap* map, const int8_t* p, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box) {
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, rank, const_cast<int8_t*>(p), dims, strides, box,
                                 es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TLR_REQUIRE(r == CUDA_SUCCESS, TLR_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}
void check16(const int8_t* p, uint64_t s1, uint64_t plane) {
  TLR_REQUIRE(reinterpret_cast<uintptr_t>(p) % 16 == 0 && s1 % 16 == 0 && plane % 16 == 0, TLR_ERR_LIMIT,
              "split product: operand not on 16-byte boundaries");
}
// Operand stored along k (element (row, k) at row * ld + k): 4D view (16 k, rows, k / 16, plane),
// box (16, box_rows, 2, 1), so that a stage holds each 16-k half as [row][16 bytes].  Rows must be
// readable (and zero) up to the next multiple of 16 past K.
void map_kmajor(CUtensorMap* map, const int8_t* p, uint64_t K, uint64_t rows, uint64_t ld, uint64_t plane,
                uint32_t box_rows) {
  check16(p, ld, plane);
  TLR_REQUIRE(K > 0 && rows > 0 && ld >= (uint64_t)oz_ld((int)K), TLR_ERR_LIMIT, "split product: bad operand shape");
  const cuuint64_t dims[4] = {16, rows, (K + 15) / 16, (cuuint64_t)OZ_S};
  const cuuint64_t strides[3] = {ld, 16, plane};
  const cuuint32_t box[4] = {16, box_rows, 2, 1};
  encode(map, p, 4, dims, strides, box);
}
// A stored along m (element (m, k) at k * ld + m): 3D view (m, k, plane), box (128, 32, 1).
void map_mmajor(CUtensorMap* map, const int8_t* p, uint64_t M, uint64_t K, uint64_t ld, uint64_t plane) {
  check16(p, ld, plane);
  TLR_REQUIRE(K > 0 && M > 0, TLR_ERR_LIMIT, "split product: bad operand shape");
  const cuuint64_t dims[3] = {M, K, (cuuint64_t)OZ_S};
  const cuuint64_t strides[2] = {ld, plane};
  const cuuint32_t box[3] = {(cuuint32_t)OZ_TM, (cuuint32_t)OZ_KS, 1};
  encode(map, p, 3, dims, strides, box);
}
}  // namespace

void oz_stats(tlr_ctx* ctx, unsigned long long out[10], int reset) {
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  TLR_CUDA(cudaMemcpyFromSymbol(out, g_oz_stats, sizeof(unsigned long long) * 10));
  if (reset) {
    const unsigned long long z[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    TLR_CUDA(cudaMemcpyToSymbol(g_oz_stats, z, sizeof(z)));
  }
}

int oz_timeout_flag(tlr_ctx* ctx) {
  int v = 0;
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  TLR_CUDA(cudaMemcpyFromSymbol(&v, g_oz_timeout, sizeof(int)));
  if (v) {
    const int zero = 0;
    TLR_CUDA(cudaMemcpyToSymbol(g_oz_timeout, &zero, sizeof(int)));
  }
  return v;
}

void oz_gemm(tlr_ctx* ctx, std::vector<OzJob>& jobs) {
  if (jobs.empty()) return;
  static bool attr = false;
  if (!attr) {
    TLR_CUDA(cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    attr = true;
  }
  // Split K per job (its shape only, so a product sums in the same order alone or in a batch):
  // enough slices of at least eight 32-deep stages for the job alone to give ~1 CTA per SM.
  int mx = 0, ny = 0;
  double flops = 0, bytes = 0;
  size_t ws_elems = 0, nctr = 0;
  for (auto& j : jobs) {
    TLR_REQUIRE(j.K > 0 && j.K <= 16384 && j.M > 0 && j.N > 0 && j.S >= 1 && j.S <= OZ_S, TLR_ERR_LIMIT,
                "split product: unsupported shape");
    const int tm = (int)oz_cdiv(j.M, OZ_TM);
    j.tiles_n = (int)oz_cdiv(j.N, OZ_TN);
    const int nst = (int)oz_cdiv(j.K, OZ_KS);
    const int tnr = j.rule_n > 0 ? (int)oz_cdiv(j.rule_n, OZ_TN) : j.tiles_n;
    const int64_t want = ((int64_t)std::max(ctx->sm_count, 1) + (int64_t)tm * tnr - 1) / ((int64_t)tm * tnr);
    if (j.nsplit <= 0) j.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({want, nst / 8, 64}));
    mx = std::max(mx, j.M);
    ny = std::max(ny, j.tiles_n * j.nsplit);
    flops += 2.0 * j.M * j.N * (double)j.K;
    // algorithmic: every chunk plane used read once, C written (and read when accumulating)
    bytes += (double)j.S * ((double)j.M * j.K + (double)j.K * j.N) + 8.0 * j.M * j.N * (j.accumulate ? 2 : 1);
    if (j.nsplit > 1) {
      ws_elems += (size_t)j.nsplit * j.M * j.N;
      nctr += (size_t)tm * j.tiles_n;
    }
  }
  double* ws = ws_elems ? static_cast<double*>(scratch(ctx, ws_elems * sizeof(double))) : nullptr;
  int* ctr = ws_elems ? split_counters(ctx, nctr) : nullptr;
  std::vector<OzDev> dev(jobs.size());
  for (size_t u = 0; u < jobs.size(); ++u) {
    const OzJob& j = jobs[u];
    OzDev& d = dev[u];
    memset(&d, 0, sizeof(d));
    const int ldb = j.ldb > 0 ? j.ldb : oz_ld(j.K);
    if (j.K0 > 0) {  // two K segments: [0, K0) from A0, [K0, K) from A
      TLR_REQUIRE(!j.acol && j.K0 % OZ_KS == 0 && j.K0 < j.K && j.A0, TLR_ERR_LIMIT,
                  "split product: bad first K segment");
      map_kmajor(&d.ta0, j.A0, (uint64_t)j.K0, (uint64_t)j.M, (uint64_t)j.lda0, j.sA0, OZ_TM);
      map_kmajor(&d.ta, j.A, (uint64_t)(j.K - j.K0), (uint64_t)j.M, (uint64_t)j.lda, j.sA, OZ_TM);
    } else if (j.acol) {
      map_mmajor(&d.ta, j.A, (uint64_t)j.M, (uint64_t)j.K, (uint64_t)j.lda, j.sA);
    } else {
      map_kmajor(&d.ta, j.A, (uint64_t)j.K, (uint64_t)j.M, (uint64_t)j.lda, j.sA, OZ_TM);
    }
    d.K0 = j.K0;
    map_kmajor(&d.tb, j.B, (uint64_t)j.K, (uint64_t)j.N, (uint64_t)ldb, j.sB, OZ_TN);
    d.eA = j.eA;
    d.eB = j.eB;
    d.C = j.C;
    d.M = j.M;
    d.N = j.N;
    d.K = j.K;
    d.ldc = j.ldc;
    d.acol = j.acol;
    d.accumulate = j.accumulate;
    d.eB_stride = j.eB_stride;
    d.nsplit = j.nsplit;
    d.tiles_n = j.tiles_n;
    d.S = j.S;
    d.tol = j.tol;
    d.smin = std::max(1, std::min(j.smin, j.S));
    if (j.nsplit > 1) {
      d.ws = ws;
      d.ctr = ctr;
      ws += (size_t)j.nsplit * j.M * j.N;
      ctr += (size_t)oz_cdiv(j.M, OZ_TM) * j.tiles_n;
    }
  }
  for (size_t o = 0; o < dev.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, dev.size() - o);
    const OzDev* dj = static_cast<const OzDev*>(upload(ctx, dev.data() + o, cnt * sizeof(OzDev)));
    if (ctx->kprof) kprof_begin(ctx);
    dim3 grid((unsigned)oz_cdiv(mx, OZ_TM), (unsigned)ny, (unsigned)cnt);
    ctx->site_next_flops = flops * cnt / jobs.size();
    TLR_SITE_PRE(ctx);
    k_oz_mma<<<grid, OZ_THREADS, OZ_SMEM, ctx->stream>>>(dj);
    TLR_LAUNCH_CHECK(ctx);
    if (ctx->kprof) kprof_end(ctx, 6, flops * cnt / jobs.size(), bytes * cnt / jobs.size());
  }
}

}  // namespace tlr
