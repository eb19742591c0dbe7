// Batched, variable-size GEMM for the TLR factorization.
//
// The paper executes the products of its sampling chains (Equation 2 / 3),
// projections (sampleLeftT), orthogonalization and dense updates as
// non-uniform batched GEMMs (Section 4.1: pointer marshaling, then a vbatched GEMM).  Here
// one launch takes an array of jobs of different shapes; each CTA computes one
// output tile of one job over its whole K range or over one slice of it
// (deterministic split-K: fixed slices, fixed-order reduction).
//
// Tile shapes follow the arithmetic units.  GB300 issues ~0.5 FP64 FMA lanes per
// SM sub-partition (SMSP) per clock, so one warp-wide DFMA occupies its SMSP's
// FP64 pipe for ~64 clocks and a single warp already saturates it: shared-memory
// bandwidth and register blocking do not matter, the number of warps with work
// does.  The FP64 instantiation therefore uses small 32 x 16 tiles (2 x 2
// outputs per thread; a 16-column right-hand side fills every warp) and splits
// long reductions so that even a single small product spreads over the 4 x 152
// SMSPs.
// FP32 FMA is 64x faster per SMSP, so the FP32 instantiation keeps 64 x 32 tiles
// with 4 x 4 outputs per thread for operand reuse.  Both stage operands through
// shared memory in 16-deep K chunks, loading chunk c + 1 into registers while
// chunk c is multiplied.
#include "common.h"

namespace tlr {

template <typename T>
struct GemmTile;
template <>
struct GemmTile<double> { static constexpr int RM = 2, RN = 2; };
template <>
struct GemmTile<float> { static constexpr int RM = 4, RN = 4; };

// 128 threads as 16 (rows) x 8 (columns); thread (tr, tc) owns rows tr*RM + i and
// columns tc*RN + j of the TM x TN tile; warp w owns columns [2w RN, 2w RN + 2 RN).
template <typename T, int MODE, int RM, int RN>
__device__ __forceinline__ void gemm_body(const GemmJob<T>* __restrict__ jobs, int njobs) {
  constexpr int TM = 16 * RM, TN_ = 8 * RN, TK = GEMM_TK;
  constexpr int EA = TK * TM / 128, EB = TK * TN_ / 128;
  // Rows padded by one where the chunk is stored across rows (consecutive threads
  // take consecutive k), which would otherwise put 16 threads on one bank.
  constexpr int PADA = (MODE == TN) ? 1 : 0, PADB = (MODE == NT) ? 0 : 1;
  __shared__ GemmJob<T> J;
  __shared__ T As[TK][TM + PADA];
  __shared__ T Bs[TK][TN_ + PADB];
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
  // Warps skip products outside the job (warp-uniform): by default warp w owns columns
  // 2w RN .. 2w RN + 2 RN - 1 of the tile (narrow N: a projection onto a few basis vectors); an
  // FP64 tile that is cut short in M (Q^T Y and Y^T Y have M = q or bs) gives warp w rows
  // 8w .. 8w+7 instead.  Either way each output is summed by one thread in k order, so the
  // mapping does not change any result.
  const bool rowwarps = (RM == 2) && (M - m0 < TM);
  const int tr = rowwarps ? ((tid >> 5) * 4 + ((tid & 31) >> 3)) : (tid & 15);
  const int tc = rowwarps ? (tid & 7) : (tid >> 4);
  const bool active = rowwarps ? (m0 + (tid >> 5) * 8 < M) : (n0 + (tid >> 5) * 2 * RN < N);
  T acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = T(0);

  // The K chunks of both segments form one sequence; this CTA takes slice [c0, c1).
  // A lower-triangular first operand contributes nothing beyond k = m0 + TM - 1.
  const int K0 = (MODE == NN && (J.flags & GEMM_ALOWER)) ? min(J.K[0], m0 + TM) : J.K[0];
  const int nch0 = (K0 + TK - 1) / TK, nch1 = J.K[1] > 0 ? (J.K[1] + TK - 1) / TK : 0;
  const int nch = nch0 + nch1;
  const int c0 = (int)((int64_t)nch * split / J.nsplit);
  const int c1 = (int)((int64_t)nch * (split + 1) / J.nsplit);
  T ra[EA], rb[EB];
  auto load = [&](int c) {
    const int seg = c < nch0 ? 0 : 1;
    const int k0 = (seg ? c - nch0 : c) * TK, K = J.K[seg];
    const T* __restrict__ A = J.A[seg];
    const T* __restrict__ B = J.B[seg];
    const int lda = J.lda[seg], ldb = J.ldb[seg];
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      const int idx = tid + e * 128;
      int m, kk;
      if (MODE == TN) { kk = idx % TK; m = idx / TK; }
      else { m = idx % TM; kk = idx / TM; }
      const int gm = m0 + m, gk = k0 + kk;
      ra[e] = (gm < M && gk < K) ? ((MODE == TN) ? A[(size_t)gk + (size_t)gm * lda] : A[(size_t)gm + (size_t)gk * lda])
                                 : T(0);
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const int idx = tid + e * 128;
      int n, kk;
      if (MODE == NT) { n = idx % TN_; kk = idx / TN_; }
      else { kk = idx % TK; n = idx / TK; }
      const int gn = n0 + n, gk = k0 + kk;
      rb[e] = (gn < N && gk < K) ? ((MODE == NT) ? B[(size_t)gn + (size_t)gk * ldb] : B[(size_t)gk + (size_t)gn * ldb])
                                 : T(0);
    }
  };
  if (c0 < c1) load(c0);
  for (int c = c0; c < c1; ++c) {
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      const int idx = tid + e * 128;
      if (MODE == TN) As[idx % TK][idx / TK] = ra[e];
      else As[idx / TM][idx % TM] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const int idx = tid + e * 128;
      if (MODE == NT) Bs[idx / TN_][idx % TN_] = rb[e];
      else Bs[idx % TK][idx / TK] = rb[e];
    }
    __syncthreads();
    if (c + 1 < c1) load(c + 1);  // in flight while this chunk is multiplied
    if (active) {
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        T a[RM], bb[RN];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = As[kk][tr * RM + i];
#pragma unroll
        for (int j = 0; j < RN; ++j) bb[j] = Bs[kk][tc * RN + j];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  const T alpha = (T)J.alpha, beta = (T)J.beta;
  if (J.nsplit == 1) {
    if (!active) return;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      const int gm = m0 + tr * RM + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        const int gn = n0 + tc * RN + j;
        if (gn >= N || ((J.flags & GEMM_TRIL) && gm < gn)) continue;
        T* c = J.C + gm + (size_t)gn * J.ldc;
        T v = alpha * acc[i][j];
        if (J.beta != 0.0) v += beta * *c;
        *c = v;
      }
    }
    return;
  }
  // Split K: store the partial; the CTA that completes the tile's set of slices
  // (arrival counter) sums all partials in slice order and writes C, then resets
  // the counter.  No CTA waits for another.  A tile strictly above the diagonal
  // of a GEMM_TRIL job returned before its first chunk in every slice, so its
  // counter is never touched.
  const size_t MN = (size_t)M * N;
  if (active) {
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      const int gm = m0 + tr * RM + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        const int gn = n0 + tc * RN + j;
        if (gn < N) J.ws[(size_t)split * MN + gm + (size_t)gn * M] = acc[i][j];
      }
    }
  }
  __threadfence();
  __syncthreads();
  __shared__ int last;
  int* ctr = J.ctr + (m0 / TM) * J.tiles_n + (n0 / TN_);
  if (tid == 0) last = (atomicAdd(ctr, 1) == J.nsplit - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Each thread sums TM*TN/128 entries side by side, so their partial loads are in flight together.
  constexpr int PER = TM * TN_ / 128;
  bool ok[PER];
  size_t o[PER];
  T v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = tid + q * 128;
    const int gm = m0 + e % TM, gn = n0 + e / TM;
    ok[q] = gm < M && gn < N && !((J.flags & GEMM_TRIL) && gm < gn);
    o[q] = ok[q] ? gm + (size_t)gn * M : 0;
    v[q] = T(0);
  }
  for (int sp = 0; sp < J.nsplit; ++sp) {
    const T* w = J.ws + (size_t)sp * MN;
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (ok[q]) v[q] += __ldcg(w + o[q]);
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (!ok[q]) continue;
    const int e = tid + q * 128;
    T* c = J.C + (m0 + e % TM) + (size_t)(n0 + e / TM) * J.ldc;
    T r = alpha * v[q];
    if (J.beta != 0.0) r += beta * *c;
    *c = r;
  }
  if (tid == 0) *ctr = 0;
}

// Job table in global memory (uploaded), for launches with many jobs.
template <typename T, int MODE, int RM, int RN>
__global__ void __launch_bounds__(128) k_gemm(const GemmJob<T>* __restrict__ jobs, int njobs) {
  gemm_body<T, MODE, RM, RN>(jobs, njobs);
}

// Job table passed as a kernel parameter (up to MAXJ jobs): no host-to-device copy ahead of the
// launch, which is most of the fixed cost of the short per-round products.
template <typename T, int MAXJ>
struct GemmParams {
  int njobs;
  GemmJob<T> jobs[MAXJ];
};
template <typename T, int MODE, int RM, int RN, int MAXJ>
__global__ void __launch_bounds__(128) k_gemm_p(const __grid_constant__ GemmParams<T, MAXJ> P) {
  gemm_body<T, MODE, RM, RN>(P.jobs, P.njobs);
}

template <typename T, int RM, int RN, int MAXJ>
static void launch_params(tlr_ctx* ctx, GemmMode mode, int64_t total, const std::vector<GemmJob<T>>& jobs) {
  GemmParams<T, MAXJ> P;
  P.njobs = (int)jobs.size();
  std::copy(jobs.begin(), jobs.end(), P.jobs);
  if (mode == NN) k_gemm_p<T, NN, RM, RN, MAXJ><<<(unsigned)total, 128, 0, ctx->stream>>>(P);
  else if (mode == TN) k_gemm_p<T, TN, RM, RN, MAXJ><<<(unsigned)total, 128, 0, ctx->stream>>>(P);
  else k_gemm_p<T, NT, RM, RN, MAXJ><<<(unsigned)total, 128, 0, ctx->stream>>>(P);
}

template <typename T>
GemmJob<T> job(GemmMode, int M, int N, const T* A, int lda, const T* B, int ldb, int K, T* C,
               int ldc, double alpha, double beta) {
  GemmJob<T> j{};
  j.A[0] = A; j.B[0] = B; j.lda[0] = lda; j.ldb[0] = ldb; j.K[0] = K;
  j.A[1] = nullptr; j.B[1] = nullptr; j.lda[1] = 1; j.ldb[1] = 1; j.K[1] = 0;
  j.C = C; j.ldc = ldc; j.M = M; j.N = N; j.alpha = alpha; j.beta = beta;
  j.flags = 0; j.ws = nullptr; j.ctr = nullptr;
  return j;
}

template <typename T>
void gemm(tlr_ctx* ctx, GemmMode mode, std::vector<GemmJob<T>>& jobs_in) {
  constexpr int RM = GemmTile<T>::RM, RN = GemmTile<T>::RN, TM = 16 * RM, TN_ = 8 * RN;
  std::vector<GemmJob<T>> jobs;
  jobs.reserve(jobs_in.size());
  for (auto& j : jobs_in)
    if (j.M > 0 && j.N > 0) jobs.push_back(j);
  if (jobs.empty()) return;
  // Split-K.  Work is counted in warp-chunks (one warp's share of a tile over one
  // 16-deep K chunk): a job has tiles_m x (warps with columns) x chunks of them.
  // Each job picks its slice length S (in chunks, at least 2) so that the job
  // alone would hold about two warps per SMSP (8 per SM), and is cut into
  // chunks / S slices, at most 64.  The choice depends on the job's own
  // shape only, never on the other jobs of the launch: a product is summed in the
  // same order whether its matrix is factored alone or in a batch, which keeps
  // batched results bitwise equal to single ones.
  const int64_t slots = 8LL * std::max(ctx->sm_count, 1);
  int64_t total = 0;
  size_t ws_elems = 0;
  std::vector<int> split_ids;
  for (size_t q = 0; q < jobs.size(); ++q) {
    auto& j = jobs[q];
    j.tiles_m = (j.M + TM - 1) / TM;
    j.tiles_n = (j.N + TN_ - 1) / TN_;
    // warps with work per tile row (columns per warp; FP64 tiles short in M: rows per warp)
    const int Nr = j.rule_n > 0 ? j.rule_n : j.N;
    int64_t wpr;
    if (RM == 2 && j.M < TM) {
      wpr = (int64_t)((j.M + 7) / 8) * ((Nr + TN_ - 1) / TN_);
    } else {
      const int full = Nr / TN_, rem = Nr % TN_;
      wpr = (int64_t)full * 4 + (rem + 2 * RN - 1) / (2 * RN);
    }
    const int chunks = (j.K[0] + GEMM_TK - 1) / GEMM_TK + (j.K[1] > 0 ? (j.K[1] + GEMM_TK - 1) / GEMM_TK : 0);
    const int64_t S = std::max<int64_t>(2, ((int64_t)j.tiles_m * wpr * chunks + slots - 1) / slots);
    j.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(64, chunks / S));
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
    size_t nctr = 0;
    for (int q : split_ids) nctr += (size_t)jobs[q].tiles_m * jobs[q].tiles_n;
    int* ctr = split_counters(ctx, nctr);
    for (int q : split_ids) {
      jobs[q].ws = ws + reinterpret_cast<size_t>(jobs[q].ws);
      jobs[q].ctr = ctr;
      ctr += (size_t)jobs[q].tiles_m * jobs[q].tiles_n;
    }
  }
  const int nj = (int)jobs.size();
  const GemmJob<T>* dj =
      nj > 64 ? static_cast<const GemmJob<T>*>(upload(ctx, jobs.data(), jobs.size() * sizeof(GemmJob<T>))) : nullptr;
  double flops = 0;
  if (ctx->kprof || ctx->site_out) {
    for (auto& j : jobs) {
      // algorithmic flops: a triangular C or a triangular A halves the product
      const double k0 = (mode == NN && (j.flags & GEMM_ALOWER)) ? 0.5 * (j.K[0] + 1) : (double)j.K[0];
      flops += 2.0 * j.M * j.N * (k0 + j.K[1]) * ((j.flags & GEMM_TRIL) ? 0.5 : 1.0);
    }
    if (ctx->kprof) kprof_begin(ctx);
  }
  ctx->site_next_flops = flops;
  TLR_SITE_PRE(ctx);
  if (nj <= 8) launch_params<T, RM, RN, 8>(ctx, mode, total, jobs);
  else if (nj <= 64) launch_params<T, RM, RN, 64>(ctx, mode, total, jobs);
  else if (mode == NN) k_gemm<T, NN, RM, RN><<<(unsigned)total, 128, 0, ctx->stream>>>(dj, nj);
  else if (mode == TN) k_gemm<T, TN, RM, RN><<<(unsigned)total, 128, 0, ctx->stream>>>(dj, nj);
  else k_gemm<T, NT, RM, RN><<<(unsigned)total, 128, 0, ctx->stream>>>(dj, nj);
  TLR_LAUNCH_CHECK(ctx);
  if (ctx->kprof) kprof_end(ctx, (sizeof(T) == 8 ? 0 : 3) + (int)mode, flops);
}

template void gemm<double>(tlr_ctx*, GemmMode, std::vector<GemmJob<double>>&);
template void gemm<float>(tlr_ctx*, GemmMode, std::vector<GemmJob<float>>&);
template GemmJob<double> job<double>(GemmMode, int, int, const double*, int, const double*, int, int,
                                     double*, int, double, double);
template GemmJob<float> job<float>(GemmMode, int, int, const float*, int, const float*, int, int,
                                   float*, int, double, double);

}  // namespace tlr
