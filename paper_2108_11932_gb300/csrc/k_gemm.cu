// Batched, variable-size GEMM for the TLR factorization.
//
// The paper executes the products of its sampling chains (Equation 2 / 3),
// projections (sampleLeftT), orthogonalization and dense updates as
// non-uniform batched GEMMs (Section 4.1, "marshaling" + vbatched GEMM).  Here
// one launch takes an array of jobs of different shapes; each CTA computes one
// 64 x 32 tile of one job over its whole K range (or over one slice of it:
// deterministic split-K with a fixed-order reduction, used when a job has few
// output tiles and a long reduction, e.g. Q^T Y with K = b).
//
// FP64 on GB300 issues ~2 DFMA per SM per clock (1.2 TFLOP/s for 152 SMs), so
// the FP64 instantiation is bound by the DFMA rate as soon as every SM holds a
// CTA: operands are staged through shared memory (coalesced 128-byte rows of
// the column-major operands) and each thread keeps a 4 x 4 register tile.
#include "common.h"

namespace tlr {

template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_gemm(const GemmJob<T>* __restrict__ jobs, int njobs) {
  constexpr int TM = GEMM_TM, TN_ = GEMM_TN, TK = GEMM_TK;
  __shared__ GemmJob<T> J;
  __shared__ T As[TK][TM];
  __shared__ T Bs[TK][TN_];
  const int tid = threadIdx.x;
  if (tid == 0) {
    int bid = blockIdx.x, lo = 0, hi = njobs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].tile0 <= bid) lo = mid; else hi = mid - 1;
    }
    J = jobs[lo];
  }
  __syncthreads();
  int local = blockIdx.x - J.tile0;
  const int split = local % J.nsplit;
  local /= J.nsplit;
  const int m0 = (local / J.tiles_n) * TM;
  const int n0 = (local % J.tiles_n) * TN_;
  if ((J.flags & GEMM_TRIL) && m0 + TM <= n0) return;  // tile strictly above the diagonal
  const int M = J.M, N = J.N;
  const int tr = tid & 15, tc = tid >> 4;
  const bool active = (n0 + (tid >> 5) * 8) < N;  // warp-uniform: this warp's 8 columns exist
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int seg = 0; seg < 2; ++seg) {
    const int K = J.K[seg];
    if (K <= 0) continue;
    const T* __restrict__ A = J.A[seg];
    const T* __restrict__ B = J.B[seg];
    const int lda = J.lda[seg], ldb = J.ldb[seg];
    const int nch = (K + TK - 1) / TK;
    const int c0 = (int)((int64_t)nch * split / J.nsplit);
    const int c1 = (int)((int64_t)nch * (split + 1) / J.nsplit);
    for (int c = c0; c < c1; ++c) {
      const int k0 = c * TK;
#pragma unroll
      for (int e = 0; e < (TK * TM) / 128; ++e) {
        const int idx = tid + e * 128;
        int m, kk;
        if (MODE == TN) { kk = idx % TK; m = idx / TK; }
        else { m = idx % TM; kk = idx / TM; }
        const int gm = m0 + m, gk = k0 + kk;
        T v = T(0);
        if (gm < M && gk < K)
          v = (MODE == TN) ? A[(size_t)gk + (size_t)gm * lda] : A[(size_t)gm + (size_t)gk * lda];
        As[kk][m] = v;
      }
#pragma unroll
      for (int e = 0; e < (TK * TN_) / 128; ++e) {
        const int idx = tid + e * 128;
        int n, kk;
        if (MODE == NT) { n = idx % TN_; kk = idx / TN_; }
        else { kk = idx % TK; n = idx / TK; }
        const int gn = n0 + n, gk = k0 + kk;
        T v = T(0);
        if (gn < N && gk < K)
          v = (MODE == NT) ? B[(size_t)gn + (size_t)gk * ldb] : B[(size_t)gk + (size_t)gn * ldb];
        Bs[kk][n] = v;
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
          T a[4], bb[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[kk][tr * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tc * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
      }
      __syncthreads();
    }
  }
  if (!active) return;
  const T alpha = (T)J.alpha, beta = (T)J.beta;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + tr * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tc * 4 + j;
      if (gn >= N) continue;
      if (J.nsplit > 1) {
        J.ws[(size_t)split * M * N + gm + (size_t)gn * M] = acc[i][j];
      } else {
        if ((J.flags & GEMM_TRIL) && gm < gn) continue;
        T* c = J.C + gm + (size_t)gn * J.ldc;
        T v = alpha * acc[i][j];
        if (J.beta != 0.0) v += beta * *c;
        *c = v;
      }
    }
  }
}

// Fixed-order reduction of split-K partials: C = alpha * sum_s ws[s] + beta * C.
template <typename T>
__global__ void k_gemm_reduce(const GemmJob<T>* __restrict__ jobs, const int* __restrict__ ids) {
  const GemmJob<T>& J = jobs[ids[blockIdx.x]];
  const size_t MN = (size_t)J.M * J.N;
  for (size_t e = blockIdx.y * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.y * blockDim.x) {
    const int gm = (int)(e % J.M), gn = (int)(e / J.M);
    T s = T(0);
    for (int sp = 0; sp < J.nsplit; ++sp) s += J.ws[(size_t)sp * MN + e];
    if ((J.flags & GEMM_TRIL) && gm < gn) continue;
    T* c = J.C + gm + (size_t)gn * J.ldc;
    T v = (T)J.alpha * s;
    if (J.beta != 0.0) v += (T)J.beta * *c;
    *c = v;
  }
}

template <typename T>
GemmJob<T> job(GemmMode, int M, int N, const T* A, int lda, const T* B, int ldb, int K, T* C,
               int ldc, double alpha, double beta) {
  GemmJob<T> j{};
  j.A[0] = A; j.B[0] = B; j.lda[0] = lda; j.ldb[0] = ldb; j.K[0] = K;
  j.A[1] = nullptr; j.B[1] = nullptr; j.lda[1] = 1; j.ldb[1] = 1; j.K[1] = 0;
  j.C = C; j.ldc = ldc; j.M = M; j.N = N; j.alpha = alpha; j.beta = beta;
  j.flags = 0; j.ws = nullptr;
  return j;
}

template <typename T>
void gemm(tlr_ctx* ctx, GemmMode mode, std::vector<GemmJob<T>>& jobs_in) {
  std::vector<GemmJob<T>> jobs;
  jobs.reserve(jobs_in.size());
  for (auto& j : jobs_in)
    if (j.M > 0 && j.N > 0) jobs.push_back(j);
  if (jobs.empty()) return;
  // Split K (deterministically: fixed slices, fixed-order reduction) when the
  // launch has fewer than ~4 CTAs per SM, so that small batches still occupy
  // every SM; each slice keeps at least 64 reduction steps.
  int64_t base = 0;
  for (auto& j : jobs) {
    j.tiles_m = (j.M + GEMM_TM - 1) / GEMM_TM;
    j.tiles_n = (j.N + GEMM_TN - 1) / GEMM_TN;
    base += (int64_t)j.tiles_m * j.tiles_n;
  }
  const int64_t target = 4LL * std::max(ctx->sm_count, 1);
  const int want = base >= target ? 1 : (int)std::min<int64_t>(16, (target + base - 1) / base);
  int64_t total = 0;
  size_t ws_elems = 0;
  std::vector<int> split_ids;
  for (size_t q = 0; q < jobs.size(); ++q) {
    auto& j = jobs[q];
    const int Kt = j.K[0] + j.K[1];
    j.nsplit = 1;
    if (!(j.flags & GEMM_TRIL) && want > 1) j.nsplit = std::max(1, std::min(want, Kt / 64));
    j.tile0 = (int)total;
    total += (int64_t)j.tiles_m * j.tiles_n * j.nsplit;
    if (j.nsplit > 1) {
      j.ws = reinterpret_cast<T*>(ws_elems);  // offset, fixed below
      ws_elems += (size_t)j.nsplit * j.M * j.N;
      split_ids.push_back((int)q);
    }
  }
  TLR_REQUIRE(total < (1LL << 31), TLR_ERR_LIMIT, "gemm: too many tiles in one launch");
  if (ws_elems) {
    T* ws = static_cast<T*>(scratch(ctx, ws_elems * sizeof(T)));
    for (int q : split_ids) jobs[q].ws = ws + reinterpret_cast<size_t>(jobs[q].ws);
  }
  const GemmJob<T>* dj =
      static_cast<const GemmJob<T>*>(upload(ctx, jobs.data(), jobs.size() * sizeof(GemmJob<T>)));
  const int nj = (int)jobs.size();
  double flops = 0;
  if (ctx->kprof) {
    for (auto& j : jobs) flops += 2.0 * j.M * j.N * (double)(j.K[0] + j.K[1]) * ((j.flags & GEMM_TRIL) ? 0.5 : 1.0);
    kprof_begin(ctx);
  }
  if (mode == NN) k_gemm<T, NN><<<(unsigned)total, 128, 0, ctx->stream>>>(dj, nj);
  else if (mode == TN) k_gemm<T, TN><<<(unsigned)total, 128, 0, ctx->stream>>>(dj, nj);
  else k_gemm<T, NT><<<(unsigned)total, 128, 0, ctx->stream>>>(dj, nj);
  TLR_LAUNCH_CHECK(ctx);
  if (ctx->kprof) kprof_end(ctx, (sizeof(T) == 8 ? 0 : 3) + (int)mode, flops);
  if (!split_ids.empty()) {
    const int* ids = static_cast<const int*>(upload(ctx, split_ids.data(), split_ids.size() * sizeof(int)));
    size_t mx = 0;
    for (int q : split_ids) mx = std::max(mx, (size_t)jobs[q].M * jobs[q].N);
    dim3 rg((unsigned)split_ids.size(), (unsigned)std::min<size_t>(64, (mx + 1023) / 1024));
    k_gemm_reduce<T><<<rg, 256, 0, ctx->stream>>>(dj, ids);
    TLR_LAUNCH_CHECK(ctx);
  }
}

template void gemm<double>(tlr_ctx*, GemmMode, std::vector<GemmJob<double>>&);
template void gemm<float>(tlr_ctx*, GemmMode, std::vector<GemmJob<float>>&);
template GemmJob<double> job<double>(GemmMode, int, int, const double*, int, const double*, int, int,
                                     double*, int, double, double);
template GemmJob<float> job<float>(GemmMode, int, int, const float*, int, const float*, int, int,
                                   float*, int, double, double);

}  // namespace tlr
