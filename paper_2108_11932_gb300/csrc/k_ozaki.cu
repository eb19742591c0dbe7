// FP64 products of the construction stage on BF16 tensor cores, exact to FP64 level.
//
// GB300 retires 2 FP64 FMAs per SM per clock but thousands of BF16 tensor-core FMAs, and
// the construction's dominant products -- the ARA samples Y = T Omega and projections
// B = T^T Q of every generated dense tile (Algorithm 1 applied to Section 6's kernel tiles)
// -- are large dense contractions.  They are computed by error-free splitting (the Ozaki
// scheme: Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012):
//
//  * Every entry x of an operand is written as x = 2^e * sum_{i=1..8} x_i 2^(-7 i) with
//    integers |x_i| <= 127, where 2^e bounds the operand block (the whole tile for T, each
//    column for Omega and Q).  The x_i are the 7-bit chunks of the 56-bit truncation of
//    |x| 2^(56-e), with the sign of x; they are found with integer operations on the FP64
//    bit pattern.  Truncation error < 2^(e-56).
//  * Each chunk is exact in BF16 (8 significant bits).  A product of chunks is an integer
//    below 2^14, and the sum of the chunk products of one pair (i, j) over 128 consecutive k,
//    even added over the (i+j-1) pairs with the same i+j, stays below 2^24: the FP32
//    accumulation of mma.sync is exact.  Every 128 k the eight group sums (i+j = 2..9) move
//    to 32-bit integer totals (exact for K <= 16384), which are combined in FP64 with weights
//    2^(-7(i+j)) once at the end; pairs with i+j > 9 are below 2^-63 of the block bounds and
//    are dropped.
//
// The error of a result entry is below ~2^-55 sum_k 2^eA 2^eB (plus FP64 rounding of the
// recombination), the same order as an FP64 dot product of the same length.
#include <cuda_bf16.h>

#include "common.h"

namespace tlr {

namespace {

constexpr int OZ_S = 8;      // slices per operand
constexpr int OZ_TM = 64;    // output rows per CTA (4 warps x 16)
constexpr int OZ_TN = 16;    // output columns per CTA (2 n8 blocks)
constexpr int OZ_KC = 32;    // k per shared-memory stage
constexpr int OZ_KF = 128;   // k per exact FP32 group sum
constexpr int OZ_LDS = 40;   // shared row stride in BF16 elements (32 + 8: conflict-free fragment loads)
constexpr int OZ_LDSM = 72;  // shared row stride of a column-oriented A chunk (64 + 8)

inline int64_t oz_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Exponent e with |x| < 2^e for the largest |x| recorded as FP64 bits (0 for an all-zero block).
__device__ __forceinline__ int oz_exponent(unsigned long long maxbits) {
  const int ex = (int)((maxbits >> 52) & 0x7FF);
  return ex == 0 ? 0 : ex - 1022;
}

// The eight signed 7-bit chunks of x relative to 2^e, as BF16 bit patterns.
__device__ __forceinline__ void oz_split(double x, int e, uint16_t out[OZ_S]) {
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
    const float f = (float)(neg ? -c : c);
    out[i] = (uint16_t)(__float_as_uint(f) >> 16);  // exact: at most 7 significant bits
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const uint16_t* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const uint16_t* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// 16-byte asynchronous global-to-shared copy; src_bytes = 0 writes zeros (the source is not read).
__device__ __forceinline__ void cp16(uint16_t* dst, const uint16_t* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

}  // namespace

// ------------------------------------------------------------------ splitting
// Slices of a batch of dense tiles (n x n each, column-major) relative to each tile's bound,
// written twice: Sc (same layout as T: row k of T^T is contiguous) and Sr (transposed: row m
// of T contiguous), so that both T Omega and T^T Q read their left operand along k.
// CTA = one 32 x 32 block of one tile; the transposed copy goes through shared memory.
__global__ void __launch_bounds__(256) k_oz_split_tiles(const double* __restrict__ T, int n,
                                                        const unsigned long long* __restrict__ tmax,
                                                        uint16_t* __restrict__ Sc, uint16_t* __restrict__ Sr,
                                                        int* __restrict__ eT) {
  const int t = blockIdx.z;
  const int e = oz_exponent(tmax[t]);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) eT[t] = e;
  const size_t n2 = (size_t)n * n;
  const double* x = T + (size_t)t * n2;
  uint16_t* oc = Sc ? Sc + (size_t)t * OZ_S * n2 : nullptr;
  uint16_t* orow = Sr + (size_t)t * OZ_S * n2;
  __shared__ uint16_t tr[OZ_S][32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int kk = ty; kk < 32; kk += 8) {
    const int m = m0 + tx, k = k0 + kk;
    uint16_t sl[OZ_S];
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

// Slices of column blocks X_j (K x ncols_j, leading dimension ld_j) relative to each
// column's bound; slice q of column c of block j lands at Xs_j + (q * ncols_j + c) * K.
// One CTA per column.
__global__ void __launch_bounds__(256) k_oz_split_cols(const OzColJob* __restrict__ jobs,
                                                       const int* __restrict__ col_job) {
  const int g = blockIdx.x;
  const OzColJob J = jobs[col_job[g]];
  const int K = J.K;
  const int c = g - J.col0;
  const double* x = J.X + (size_t)c * J.ld;
  const int ldo = J.ldo > 0 ? J.ldo : K;
  const size_t plane = J.plane > 0 ? J.plane : (size_t)J.ncols * ldo;
  uint16_t* xs = J.Xs + (size_t)c * ldo;
  if (J.efix != OZ_EFIX_NONE || J.emax) {
    const int e = J.emax ? oz_exponent(*J.emax) : J.efix;
    if (J.emax && J.e && c == 0 && threadIdx.x == 0) J.e[0] = e;
    for (int k = threadIdx.x; k < ldo; k += blockDim.x) {
      uint16_t s[OZ_S];
      if (k < K) oz_split(x[k], e, s);
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) xs[(size_t)q * plane + k] = k < K ? s[q] : (uint16_t)0;
    }
    return;
  }
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
  const int e = oz_exponent(red[0]);
  if (threadIdx.x == 0) J.e[c] = e;
  for (int k = threadIdx.x; k < ldo; k += blockDim.x) {
    uint16_t s[OZ_S];
    if (k < K) oz_split(x[k], e, s);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) xs[(size_t)q * plane + k] = k < K ? s[q] : (uint16_t)0;
  }
}

// ------------------------------------------------------------------ product
// C(M x N) = 2^(eA + eB_c) * sum over slice pairs (i, j), i + j <= 9, of A_i B_j 2^(-7(i+j)):
// A(m, k) = A_i[k + m * lda] (rows of A contiguous along k), B(k, n) = B_j[k + n * K].
// K and lda are multiples of 8 (16-byte rows).  Grid (M / 64, N / 16, jobs); warp w owns
// rows 16w .. 16w+15 of the CTA's 64 x 16 block.
template <bool ACOL>
__global__ void __launch_bounds__(128) k_oz_gemm(const OzJob* __restrict__ jobs) {
  const OzJob J = jobs[blockIdx.z];
  if ((int)blockIdx.y >= J.tiles_n * J.nsplit) return;
  const int nt = blockIdx.y % J.tiles_n, split = blockIdx.y / J.tiles_n;
  const int m0 = blockIdx.x * OZ_TM, n0 = nt * OZ_TN;
  if (m0 >= J.M || n0 >= J.N) return;
  extern __shared__ __align__(16) uint16_t oz_sm[];
  constexpr int STAGE = OZ_S * (OZ_TM + OZ_TN) * OZ_LDS;  // elements per buffer
  // two buffers, each [slice][row 64][k 32 (+8)] (A) then [slice][col 16][k 32 (+8)] (B)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int M = J.M, N = J.N, K = J.K;
  float acc[OZ_S][2][4];  // exact group sums of the current 128-k window (integers < 2^24)
  int tot[OZ_S][2][4];    // exact group sums over all k so far (integers < 2^31 for K <= 16384)
#pragma unroll
  for (int g = 0; g < OZ_S; ++g)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc[g][j][r] = 0.f;
        tot[g][j][r] = 0;
      }
  // ldmatrix row addresses: A matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15); B matrices
  // (columns 0-7 | 8-15) x (k 0-7 | 8-15) of the CTA's 16 columns
  const int mi = lane >> 3, ri = lane & 7;
  // row-oriented A chunk [slice][row][k]: matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15);
  // column-oriented [slice][k][row]: the same four matrices read transposed
  const int a_off = ACOL ? ((mi >> 1) * 8 + ri) * OZ_LDSM + warp * 16 + (mi & 1) * 8
                         : (warp * 16 + ri + (mi & 1) * 8) * OZ_LDS + (mi >> 1) * 8;
  const int a_slice = ACOL ? OZ_KC * OZ_LDSM : OZ_TM * OZ_LDS;  // elements per slice of a chunk
  const int a_ks = ACOL ? OZ_LDSM : 1;                          // step of k within a chunk
  const int ldb = J.ldb > 0 ? J.ldb : K;
  const int b_off = OZ_S * OZ_TM * OZ_LDS + (ri + (mi >> 1) * 8) * OZ_LDS + (mi & 1) * 8;
  // copy chunk k0 (16-byte pieces of 8 consecutive k) into buffer `buf`, zero-filled outside
  auto stage = [&](int k0, int buf) {
    uint16_t* As = oz_sm + buf * STAGE;
    uint16_t* Bs = As + OZ_S * OZ_TM * OZ_LDS;
    if (ACOL) {  // pieces of 8 consecutive rows at one k
      for (int e = tid; e < OZ_S * OZ_KC * 8; e += 128) {
        const int p = e & 7, kk = (e >> 3) & (OZ_KC - 1), q = e / (8 * OZ_KC);
        const int gm = m0 + 8 * p, gk = k0 + kk;
        const bool in = gm < M && gk < K;
        cp16(As + (q * OZ_KC + kk) * OZ_LDSM + 8 * p, in ? J.A + (size_t)q * J.sA + gm + (size_t)gk * J.lda : J.A,
             in ? 16 : 0);
      }
    } else {  // pieces of 8 consecutive k in one row
      for (int e = tid; e < OZ_S * OZ_TM * 4; e += 128) {
        const int p = e & 3, r = (e >> 2) % OZ_TM, q = e / (4 * OZ_TM);
        const int gm = m0 + r, gk = k0 + 8 * p;
        const bool in = gm < M && gk < K;
        cp16(As + (q * OZ_TM + r) * OZ_LDS + 8 * p, in ? J.A + (size_t)q * J.sA + gk + (size_t)gm * J.lda : J.A,
             in ? 16 : 0);
      }
    }
    for (int e = tid; e < OZ_S * OZ_TN * 4; e += 128) {
      const int p = e & 3, c = (e >> 2) % OZ_TN, q = e / (4 * OZ_TN);
      const int gn = n0 + c, gk = k0 + 8 * p;
      const bool in = gn < N && gk < K;
      cp16(Bs + (q * OZ_TN + c) * OZ_LDS + 8 * p, in ? J.B + (size_t)q * J.sB + gk + (size_t)gn * ldb : J.B,
           in ? 16 : 0);
    }
    cp_commit();
  };
  const int nch = (K + OZ_KC - 1) / OZ_KC;
  const int kb = (int)((int64_t)nch * split / J.nsplit) * OZ_KC;
  const int ke = min(K, (int)((int64_t)nch * (split + 1) / J.nsplit) * OZ_KC);
  if (kb < ke) stage(kb, 0);
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += OZ_KC, buf ^= 1) {
    if (k0 + OZ_KC < ke) {
      stage(k0 + OZ_KC, buf ^ 1);  // next chunk in flight while this one is multiplied
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const uint16_t* base = oz_sm + buf * STAGE;
#pragma unroll
    for (int ks = 0; ks < OZ_KC; ks += 16) {
      uint32_t b[OZ_S][4];  // per slice j: b0, b1 of columns 0-7, then of columns 8-15
#pragma unroll
      for (int j = 0; j < OZ_S; ++j) ldsm_x4(b[j], base + b_off + j * OZ_TN * OZ_LDS + ks);
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        uint32_t a[4];
        if (ACOL) ldsm_x4_t(a, base + a_off + i * a_slice + ks * a_ks);
        else ldsm_x4(a, base + a_off + i * a_slice + ks * a_ks);
#pragma unroll
        for (int j = 0; j + i < OZ_S; ++j) {
          mma_bf16(acc[i + j][0], a[0], a[1], a[2], a[3], b[j][0], b[j][1]);
          mma_bf16(acc[i + j][1], a[0], a[1], a[2], a[3], b[j][2], b[j][3]);
        }
      }
    }
    __syncthreads();
    if (((k0 + OZ_KC - kb) % OZ_KF) == 0 || k0 + OZ_KC >= ke) {  // move the exact window sums to integers
#pragma unroll
      for (int g = 0; g < OZ_S; ++g)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            tot[g][nb][r] += __float2int_rn(acc[g][nb][r]);
            acc[g][nb][r] = 0.f;
          }
    }
  }
  const int eA = *J.eA;
  const size_t MN = (size_t)M * N;
#pragma unroll
  for (int nb = 0; nb < 2; ++nb)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gm = m0 + warp * 16 + gq + ((r & 2) ? 8 : 0);
      const int gn = n0 + nb * 8 + 2 * tq + (r & 1);
      if (gm < M && gn < N) {
        double v = 0.0;  // smallest weights first
#pragma unroll
        for (int g = OZ_S - 1; g >= 0; --g) v = fma((double)tot[g][nb][r], ldexp(1.0, -7 * (g + 2)), v);
        v = ldexp(v, eA + J.eB[gn * J.eB_stride]);
        if (J.nsplit > 1) {
          J.ws[(size_t)split * MN + gm + (size_t)gn * M] = v;
        } else {
          double* c = J.C + gm + (size_t)gn * J.ldc;
          *c = J.accumulate ? *c + v : v;
        }
      }
    }
  if (J.nsplit == 1) return;
  // the last slice to finish this output block sums the partials in slice order
  __threadfence();
  __syncthreads();
  __shared__ int last;
  int* ctr = J.ctr + (m0 / OZ_TM) * J.tiles_n + nt;
  if (tid == 0) last = (atomicAdd(ctr, 1) == J.nsplit - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = tid; e < OZ_TM * OZ_TN; e += 128) {
    const int gm = m0 + e % OZ_TM, gn = n0 + e / OZ_TM;
    if (gm >= M || gn >= N) continue;
    const size_t o = gm + (size_t)gn * M;
    double v = 0.0;
    for (int sp = 0; sp < J.nsplit; ++sp) v += __ldcg(J.ws + (size_t)sp * MN + o);
    double* c = J.C + gm + (size_t)gn * J.ldc;
    *c = J.accumulate ? *c + v : v;
  }
  if (tid == 0) *ctr = 0;
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

static size_t oz_gemm_smem() { return 2 * sizeof(uint16_t) * OZ_S * (OZ_TM + OZ_TN) * OZ_LDS; }

void oz_split_tiles(tlr_ctx* ctx, int ntiles, int n, const double* T, const unsigned long long* tmax, uint16_t* Sc,
                    uint16_t* Sr, int* eT) {
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

void oz_gemm(tlr_ctx* ctx, std::vector<OzJob>& jobs) {
  if (jobs.empty()) return;
  static bool attr = false;
  if (!attr) {
    TLR_CUDA(cudaFuncSetAttribute(k_oz_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_gemm_smem()));
    TLR_CUDA(cudaFuncSetAttribute(k_oz_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_gemm_smem()));
    attr = true;
  }
  const bool acol = jobs[0].acol != 0;
  for (auto& j : jobs) {
    const int ldb = j.ldb > 0 ? j.ldb : j.K;
    // 16-byte pieces: rows of A (or its columns), columns of B, all on 8-element boundaries
    TLR_REQUIRE((j.acol != 0) == acol && j.lda % 8 == 0 && ldb % 8 == 0 && j.K <= 16384 &&
                    (acol ? j.M % 8 == 0 : j.K % 8 == 0),
                TLR_ERR_LIMIT, "split product: unsupported shape");
  }
  // Split K per job (its shape only, so a product sums in the same order alone or in a batch):
  // enough slices of at least eight 32-deep chunks for the job alone to give ~1 CTA per SM.
  int mx = 0, ny = 0;
  double flops = 0;
  size_t ws_elems = 0, nctr = 0;
  for (auto& j : jobs) {
    const int tm = (j.M + OZ_TM - 1) / OZ_TM;
    j.tiles_n = (j.N + OZ_TN - 1) / OZ_TN;
    const int nch = (j.K + OZ_KC - 1) / OZ_KC;
    const int tnr = j.rule_n > 0 ? (j.rule_n + OZ_TN - 1) / OZ_TN : j.tiles_n;
    const int64_t want = ((int64_t)std::max(ctx->sm_count, 1) + (int64_t)tm * tnr - 1) / ((int64_t)tm * tnr);
    if (j.nsplit <= 0) j.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({want, nch / 8, 64}));
    mx = std::max(mx, j.M);
    ny = std::max(ny, j.tiles_n * j.nsplit);
    flops += 2.0 * j.M * j.N * (double)j.K;
    if (j.nsplit > 1) {
      ws_elems += (size_t)j.nsplit * j.M * j.N;
      nctr += (size_t)tm * j.tiles_n;
    }
  }
  if (ws_elems) {
    double* ws = static_cast<double*>(scratch(ctx, ws_elems * sizeof(double)));
    int* ctr = split_counters(ctx, nctr);
    for (auto& j : jobs)
      if (j.nsplit > 1) {
        j.ws = ws;
        j.ctr = ctr;
        ws += (size_t)j.nsplit * j.M * j.N;
        ctr += (size_t)((j.M + OZ_TM - 1) / OZ_TM) * j.tiles_n;
      }
  }
  double bytes = 0;  // algorithmic: every slice read once, C written (and read when accumulating)
  for (auto& j : jobs)
    bytes += 16.0 * j.M * j.K + 16.0 * j.K * j.N + 8.0 * j.M * j.N * (j.accumulate ? 2 : 1);
  for (size_t o = 0; o < jobs.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, jobs.size() - o);
    const OzJob* dj = static_cast<const OzJob*>(upload(ctx, jobs.data() + o, cnt * sizeof(OzJob)));
    if (ctx->kprof) kprof_begin(ctx);
    dim3 grid((unsigned)oz_cdiv(mx, OZ_TM), (unsigned)ny, (unsigned)cnt);
    ctx->site_next_flops = flops * cnt / jobs.size();
    TLR_SITE_PRE(ctx);
    if (acol) k_oz_gemm<true><<<grid, 128, oz_gemm_smem(), ctx->stream>>>(dj);
    else k_oz_gemm<false><<<grid, 128, oz_gemm_smem(), ctx->stream>>>(dj);
    TLR_LAUNCH_CHECK(ctx);
    if (ctx->kprof) kprof_end(ctx, 6, flops * cnt / jobs.size(), bytes * cnt / jobs.size());
  }
}

}  // namespace tlr
