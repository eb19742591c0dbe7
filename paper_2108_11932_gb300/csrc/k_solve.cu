// Skinny batched products of the TLR triangular solves (Algorithm 7 and its transpose).
//
// A solve with a few right-hand sides multiplies every stored factor block (L_kk^-1, U_ik, V_ik) by a
// block of nrhs <= 32 columns: one or a few FP64 FMAs per matrix entry read.  The tile GEMM (32 x 16
// outputs per CTA) would pad nrhs = 1 to 16 columns, i.e. 16 times the FP64 work; here each thread
// keeps NR <= 8 columns in registers and the matrix is read once per group of NR columns, so the
// kernels run at the FP64 FMA rate (one FMA per 8 bytes for nrhs = 1 is ~0.85 TFMA/s of HBM
// bandwidth against ~0.63 TFMA/s of DFMA) without padding.  Sums are reduced in a fixed order (no
// atomics): results do not depend on timing.
#include <algorithm>

#include "common.h"

namespace tlr {

constexpr int SK_THREADS = 256;
// k steps whose loads are issued together (as many as the registers of NR accumulators allow)
template <int NR>
struct SkUnroll {
  static constexpr int U = NR <= 2 ? 8 : 4;
};

__device__ __forceinline__ void sk_store(const SkJob& J, int m, int n, double v) {
  double* c = J.C + m + (size_t)n * J.ldc;
  *c = J.beta == 0.0 ? J.alpha * v : fma(J.alpha, v, J.beta * *c);
}

// C = alpha A B + beta C, A column-major (M x K).  One CTA per work item (job, first row m0, 2^ks_log2
// k-slots): 256 / KS rows x KS k-slots, thread (row, slot) sums k = slot, slot + KS, ...; the slot sums
// of an output are added in slot order.  Items are made per job from its K (at most 8 steps per slot
// up to 64 slots), so short and long products alike fill a launch.  lower: A(m, k) = 0 for k > m.
template <int NR>
__global__ void __launch_bounds__(SK_THREADS) k_sk_nn(const SkJob* __restrict__ jobs, const SkItem* __restrict__ items,
                                                      int nrhs) {
  constexpr int SK_U = SkUnroll<NR>::U;
  const SkItem it = items[blockIdx.x];
  const SkJob J = jobs[it.job];
  __shared__ double red[SK_THREADS][NR];
  const int KS = 1 << it.cfg, rb = SK_THREADS >> it.cfg;
  const int t = threadIdx.x, r = t & (rb - 1), ks = t >> (8 - it.cfg);
  const int m = it.m0 + r;
  const int kend = m < J.M ? (J.lower ? min(J.K, m + 1) : J.K) : 0;
  for (int n0 = 0; n0 < nrhs; n0 += NR) {
    const int nn = min(NR, nrhs - n0);
    double acc[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) acc[i] = 0.0;
    const double* B = J.B + (size_t)n0 * J.ldb;
    int k = ks;
    for (; k + (SK_U - 1) * KS < kend; k += SK_U * KS) {  // SK_U independent loads in flight
      double a[SK_U], bv[SK_U][NR];
#pragma unroll
      for (int u = 0; u < SK_U; ++u) {
        a[u] = J.A[m + (size_t)(k + u * KS) * J.lda];
#pragma unroll
        for (int i = 0; i < NR; ++i) bv[u][i] = i < nn ? __ldg(B + k + u * KS + (size_t)i * J.ldb) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < SK_U; ++u)
#pragma unroll
        for (int i = 0; i < NR; ++i) acc[i] = fma(a[u], bv[u][i], acc[i]);
    }
    for (; k < kend; k += KS) {
      const double a = J.A[m + (size_t)k * J.lda];
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if (i < nn) acc[i] = fma(a, __ldg(B + k + (size_t)i * J.ldb), acc[i]);
    }
    if (KS == 1) {
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if (i < nn && m < J.M) sk_store(J, m, n0 + i, acc[i]);
      continue;
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) red[t][i] = acc[i];
    __syncthreads();
    for (int o = t; o < rb * nn; o += SK_THREADS) {
      const int rr = o % rb, i = o / rb;
      if (it.m0 + rr < J.M) {
        double v = 0.0;
        for (int q = 0; q < KS; ++q) v += red[q * rb + rr][i];
        sk_store(J, it.m0 + rr, n0 + i, v);
      }
    }
    __syncthreads();
  }
}

// C = alpha A^T B + beta C, A column-major (K x M): one warp per output row m (a column of A), 8 rows
// per work item, lanes along k, butterfly sums.  lower: A is lower triangular, so column m is zero
// above row m.
template <int NR>
__global__ void __launch_bounds__(SK_THREADS) k_sk_tn(const SkJob* __restrict__ jobs, const SkItem* __restrict__ items,
                                                      int nrhs) {
  constexpr int SK_U = SkUnroll<NR>::U;
  const SkItem it = items[blockIdx.x];
  const SkJob J = jobs[it.job];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = it.m0 + warp;
  if (m >= J.M) return;
  const double* a = J.A + (size_t)m * J.lda;
  const int kb = J.lower ? (m & ~31) : 0;
  for (int n0 = 0; n0 < nrhs; n0 += NR) {
    const int nn = min(NR, nrhs - n0);
    double acc[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) acc[i] = 0.0;
    const double* B = J.B + (size_t)n0 * J.ldb;
    int k = kb + lane;
    for (; k + (SK_U - 1) * 32 < J.K; k += SK_U * 32) {  // SK_U independent loads in flight
      double av[SK_U], bv[SK_U][NR];
#pragma unroll
      for (int u = 0; u < SK_U; ++u) {
        av[u] = a[k + u * 32];
#pragma unroll
        for (int i = 0; i < NR; ++i) bv[u][i] = i < nn ? B[k + u * 32 + (size_t)i * J.ldb] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < SK_U; ++u)
#pragma unroll
        for (int i = 0; i < NR; ++i) acc[i] = fma(av[u], bv[u][i], acc[i]);
    }
    for (; k < J.K; k += 32) {
      const double av = a[k];
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if (i < nn) acc[i] = fma(av, B[k + (size_t)i * J.ldb], acc[i]);
    }
#pragma unroll
    for (int i = 0; i < NR; ++i)
      for (int o = 16; o; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    double mine = 0.0;
#pragma unroll
    for (int i = 0; i < NR; ++i)
      if (lane == i) mine = acc[i];
    if (lane < nn) sk_store(J, m, n0 + lane, mine);
  }
}

void sk_items(int tn, const std::vector<SkJob>& jobs, int job0, std::vector<SkItem>& items) {
  for (size_t q = 0; q < jobs.size(); ++q) {
    const SkJob& J = jobs[q];
    int cfg = 0;  // log2 of the k-slots: at most 8 k steps per slot, at most 64 slots (4 rows)
    if (!tn)
      while (cfg < 6 && ((J.K + (1 << cfg) - 1) >> cfg) > 8) ++cfg;
    const int rows = tn ? SK_THREADS / 32 : SK_THREADS >> cfg;
    for (int m0 = 0; m0 < J.M; m0 += rows) items.push_back(SkItem{job0 + (int)q, m0, cfg});
  }
}

template <int NR>
static void sk_launch(tlr_ctx* ctx, int tn, const SkJob* jobs, const SkItem* items, int nitems, int nrhs) {
  if (tn) {
    k_sk_tn<NR><<<(unsigned)nitems, SK_THREADS, 0, ctx->stream>>>(jobs, items, nrhs);
    TLR_LAUNCH_CHECK(ctx);
  } else {
    k_sk_nn<NR><<<(unsigned)nitems, SK_THREADS, 0, ctx->stream>>>(jobs, items, nrhs);
    TLR_LAUNCH_CHECK(ctx);
  }
}

void sk_gemm(tlr_ctx* ctx, int tn, const SkJob* jobs, const SkItem* items, int nitems, int nrhs) {
  if (nitems <= 0 || nrhs <= 0) return;
  TLR_SITE_PRE(ctx);
  if (nrhs == 1) sk_launch<1>(ctx, tn, jobs, items, nitems, nrhs);
  else if (nrhs == 2) sk_launch<2>(ctx, tn, jobs, items, nitems, nrhs);
  else if (nrhs <= 4) sk_launch<4>(ctx, tn, jobs, items, nitems, nrhs);
  else sk_launch<8>(ctx, tn, jobs, items, nitems, nrhs);
}

// ------------------------------------------------------------------ preconditioned CG vectors
// out[c] = sum_i X(i, c) Y(i, c): one CTA per column, strided partial sums, then a fixed-order tree.
__global__ void __launch_bounds__(256) k_coldot(int64_t n, const double* __restrict__ X, int64_t ldx,
                                                const double* __restrict__ Y, int64_t ldy, double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  const double* x = X + (size_t)c * ldx;
  const double* y = Y + (size_t)c * ldy;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s = fma(x[i], y[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

void coldot(tlr_ctx* ctx, int64_t n, int ncols, const double* X, int64_t ldx, const double* Y, int64_t ldy,
            double* out) {
  if (ncols <= 0) return;
  TLR_SITE_PRE(ctx);
  k_coldot<<<(unsigned)ncols, 256, 0, ctx->stream>>>(n, X, ldx, Y, ldy, out);
  TLR_LAUNCH_CHECK(ctx);
}

// Active columns c (active[c] != 0): x += a p, r -= a q with a = num[c] / den[c].
__global__ void k_pcg_xr(int64_t n, const double* __restrict__ num, const double* __restrict__ den,
                         const int* __restrict__ active, double* __restrict__ x, int64_t ldx,
                         const double* __restrict__ p, double* __restrict__ r, const double* __restrict__ q,
                         int64_t ld) {
  const int c = blockIdx.y;
  if (!active[c]) return;
  const double a = num[c] / den[c];
  const size_t o = (size_t)c * ld;
  double* xc = x + (size_t)c * ldx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    xc[i] = fma(a, p[o + i], xc[i]);
    r[o + i] = fma(-a, q[o + i], r[o + i]);
  }
}

// Active columns: p = z + b p with b = num[c] / den[c].
__global__ void k_pcg_p(int64_t n, const double* __restrict__ num, const double* __restrict__ den,
                        const int* __restrict__ active, const double* __restrict__ z, double* __restrict__ p,
                        int64_t ld) {
  const int c = blockIdx.y;
  if (!active[c]) return;
  const double bt = num[c] / den[c];
  const size_t o = (size_t)c * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[o + i] = fma(bt, p[o + i], z[o + i]);
}

void pcg_update_xr(tlr_ctx* ctx, int64_t n, int ncols, const double* num, const double* den, const int* active,
                   double* x, int64_t ldx, const double* p, double* r, const double* q, int64_t ld) {
  if (ncols <= 0 || n <= 0) return;
  const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  TLR_SITE_PRE(ctx);
  k_pcg_xr<<<dim3(gx, (unsigned)ncols), 256, 0, ctx->stream>>>(n, num, den, active, x, ldx, p, r, q, ld);
  TLR_LAUNCH_CHECK(ctx);
}

void pcg_update_p(tlr_ctx* ctx, int64_t n, int ncols, const double* num, const double* den, const int* active,
                  const double* z, double* p, int64_t ld) {
  if (ncols <= 0 || n <= 0) return;
  const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  TLR_SITE_PRE(ctx);
  k_pcg_p<<<dim3(gx, (unsigned)ncols), 256, 0, ctx->stream>>>(n, num, den, active, z, p, ld);
  TLR_LAUNCH_CHECK(ctx);
}

}  // namespace tlr
