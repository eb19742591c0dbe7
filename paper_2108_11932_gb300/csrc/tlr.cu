// Host side of the GB300 TLR library: context and memory, the batched ARA
// engine with dynamic batching (Algorithm 1 + Algorithm 5), TLR construction,
// left-looking TLR Cholesky / LDL^T (Algorithm 6 / Algorithm 10), TLR solve
// (Algorithm 7), log-determinant, products, and the C ABI.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <numeric>

#include "common.h"

using namespace tlr;

namespace tlr {

// ======================================================================== memory
void* dalloc(tlr_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, ctx->user);
    TLR_REQUIRE(p != nullptr, TLR_ERR_NOMEM, "device allocation failed");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(TLR_ERR_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
  }
  return p;
}

void dfree(tlr_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->free_fn) ctx->free_fn(p, ctx->user);
  else cudaFreeAsync(p, ctx->stream);
}

// Split-K scratch; each stream has its own so that overlapped launches never share it.
void* scratch(tlr_ctx* ctx, size_t bytes) {
  const bool side = ctx->side && ctx->stream == ctx->side;
  void*& p = side ? ctx->scratch_side : ctx->scratch;
  size_t& cap = side ? ctx->scratch_side_cap : ctx->scratch_cap;
  if (bytes > cap) {
    if (side) TLR_CUDA(cudaStreamSynchronize(ctx->side));  // the old buffer may still be read
    dfree(ctx, p);
    p = nullptr;
    const size_t ncap = std::max(bytes, cap * 2);
    cap = 0;
    p = dalloc(ctx, ncap);
    cap = ncap;
  }
  return p;
}

// Job descriptors travel through a pinned staging ring mirrored on the device.
// Before the ring wraps the stream is synchronized, so no launch still reads
// the region being overwritten.
void* upload(tlr_ctx* ctx, const void* host, size_t bytes) {
  const size_t need = (bytes + 255) & ~size_t(255);
  TLR_REQUIRE(need <= ctx->ring_cap, TLR_ERR_LIMIT, "job list larger than the upload ring");
  if (ctx->ring_pos + need > ctx->ring_cap) {
    // no launch on either stream may still read the region about to be reused
    TLR_CUDA(cudaStreamSynchronize(ctx->main));
    if (ctx->side) TLR_CUDA(cudaStreamSynchronize(ctx->side));
    ctx->ring_pos = 0;
  }
  char* h = ctx->pinned + ctx->ring_pos;
  char* d = ctx->djobs + ctx->ring_pos;
  memcpy(h, host, bytes);
  TLR_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, ctx->stream));
  ctx->ring_pos += need;
  return d;
}

void* host_status(tlr_ctx* ctx, size_t bytes) {
  if (bytes > ctx->hstatus_cap) {
    if (ctx->hstatus) cudaFreeHost(ctx->hstatus);
    ctx->hstatus = nullptr;
    TLR_CUDA(cudaMallocHost(&ctx->hstatus, bytes));
    ctx->hstatus_cap = bytes;
  }
  return ctx->hstatus;
}

void prof_mark(tlr_ctx* ctx, int phase) {
  if (!ctx->prof) return;
  if (ctx->cur_phase >= 0) ctx->phase_launch[ctx->cur_phase] += ctx->launches - ctx->phase_launch0;
  ctx->phase_launch0 = ctx->launches;
  ctx->cur_phase = phase;
  if (ctx->ev_n == ctx->ev.size()) {
    cudaEvent_t e;
    TLR_CUDA(cudaEventCreate(&e));
    ctx->ev.push_back(e);
    ctx->ev_phase.push_back(0);
  }
  TLR_CUDA(cudaEventRecord(ctx->ev[ctx->ev_n], ctx->stream));
  ctx->ev_phase[ctx->ev_n] = phase;
  ctx->ev_n++;
}

void prof_flush(tlr_ctx* ctx) {
  if (!ctx->prof || ctx->ev_n == 0) return;
  prof_mark(ctx, PH_OTHER);
  TLR_CUDA(cudaStreamSynchronize(ctx->main));
  if (ctx->side) TLR_CUDA(cudaStreamSynchronize(ctx->side));
  for (size_t e = 0; e + 1 < ctx->ev_n; ++e) {
    float ms = 0;
    TLR_CUDA(cudaEventElapsedTime(&ms, ctx->ev[e], ctx->ev[e + 1]));
    ctx->phase_ms[ctx->ev_phase[e]] += ms;
  }
  ctx->ev_n = 0;
  ctx->cur_phase = -1;
}

void kprof_begin(tlr_ctx* ctx) {
  while (ctx->kev.size() < ctx->kev_n + 2) {
    cudaEvent_t e;
    TLR_CUDA(cudaEventCreate(&e));
    ctx->kev.push_back(e);
  }
  if (ctx->kev_fam.size() < ctx->kev.size()) {
    ctx->kev_fam.resize(ctx->kev.size());
    ctx->kev_flops.resize(ctx->kev.size());
  }
  TLR_CUDA(cudaEventRecord(ctx->kev[ctx->kev_n], ctx->stream));
}

void kprof_end(tlr_ctx* ctx, int family, double flops) {
  TLR_CUDA(cudaEventRecord(ctx->kev[ctx->kev_n + 1], ctx->stream));
  ctx->kev_fam[ctx->kev_n] = family;
  ctx->kev_flops[ctx->kev_n] = flops;
  ctx->kev_n += 2;
  if (ctx->kev_n >= 16384) kprof_flush(ctx);
}

void kprof_flush(tlr_ctx* ctx) {
  if (ctx->kev_n == 0) return;
  TLR_CUDA(cudaStreamSynchronize(ctx->main));  // events may sit on either stream
  if (ctx->side) TLR_CUDA(cudaStreamSynchronize(ctx->side));
  for (size_t e = 0; e < ctx->kev_n; e += 2) {
    float ms = 0;
    TLR_CUDA(cudaEventElapsedTime(&ms, ctx->kev[e], ctx->kev[e + 1]));
    const int f = ctx->kev_fam[e];
    ctx->kfam_ms[f] += ms;
    ctx->kfam_flops[f] += ctx->kev_flops[e];
    ctx->kfam_launches[f] += 1;
  }
  ctx->kev_n = 0;
}

// Grow-only device workspace.
struct Buf {
  tlr_ctx* ctx = nullptr;
  void* p = nullptr;
  size_t cap = 0;
  explicit Buf(tlr_ctx* c) : ctx(c) {}
  ~Buf() { dfree(ctx, p); }
  template <typename T>
  T* need(size_t elems) {
    const size_t bytes = std::max<size_t>(elems * sizeof(T), 256);
    if (bytes > cap) {
      dfree(ctx, p);
      p = nullptr;
      cap = 0;
      p = dalloc(ctx, bytes + bytes / 4);
      cap = bytes + bytes / 4;
    }
    return static_cast<T*>(p);
  }
};

static void d2h_sync(tlr_ctx* ctx, void* host, const void* dev, size_t bytes) {
  TLR_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->prof) {
    const auto t0 = std::chrono::steady_clock::now();
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->host_wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  } else {
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  }
}

// ======================================================================== dense diagonal tiles
constexpr int NBK = 64;

// Blocked right-looking Cholesky / unpivoted LDL^T of an n x n tile (lower).
// info (device int) must hold -1 on entry; receives the first failing column.
static void dense_factor(tlr_ctx* ctx, int n, double* A, int lda, int ldl, double* dvec, int* info,
                         Buf& tmp) {
  for (int p = 0; p < n; p += NBK) {
    const int pb = std::min(NBK, n - p);
    double* App = A + p + (size_t)p * lda;
    potrf_diag_block(ctx, pb, App, lda, ldl, dvec, info, p);
    const int m = n - p - pb;
    if (m <= 0) continue;
    double* P = A + (p + pb) + (size_t)p * lda;
    trsm_panel_right(ctx, m, pb, App, lda, P, lda, ldl, ldl ? dvec + p : nullptr);
    const double* Pl = P;
    int ldpl = lda;
    if (ldl) {
      double* W = tmp.need<double>((size_t)m * pb);
      scale_cols(ctx, m, pb, dvec + p, P, lda, W, m);
      Pl = W;
      ldpl = m;
    }
    std::vector<GemmJob<double>> jobs{job<double>(NT, m, m, Pl, ldpl, P, lda, pb,
                                                  A + (p + pb) + (size_t)(p + pb) * lda, lda, -1.0, 1.0)};
    jobs[0].flags = GEMM_TRIL;
    gemm<double>(ctx, NT, jobs);
  }
}

// X = L^{-1} X (trans = 0) or X = L^{-T} X (trans = 1), L n x n lower.
static void dense_trsm(tlr_ctx* ctx, int n, const double* L, int lda, int unit, int nrhs, double* X,
                       int ldx, int trans) {
  if (nrhs <= 0) return;
  if (!trans) {
    for (int p = 0; p < n; p += NBK) {
      const int pb = std::min(NBK, n - p);
      trsm_left_block(ctx, pb, L + p + (size_t)p * lda, lda, unit, nrhs, X + p, ldx);
      const int m = n - p - pb;
      if (m > 0) {
        std::vector<GemmJob<double>> jobs{job<double>(NN, m, nrhs, L + (p + pb) + (size_t)p * lda, lda,
                                                      X + p, ldx, pb, X + p + pb, ldx, -1.0, 1.0)};
        gemm<double>(ctx, NN, jobs);
      }
    }
  } else {
    const int last = ((n - 1) / NBK) * NBK;
    for (int p = last; p >= 0; p -= NBK) {
      const int pb = std::min(NBK, n - p);
      const int m = n - p - pb;
      if (m > 0) {
        std::vector<GemmJob<double>> jobs{job<double>(TN, pb, nrhs, L + (p + pb) + (size_t)p * lda, lda,
                                                      X + p + pb, ldx, m, X + p, ldx, -1.0, 1.0)};
        gemm<double>(ctx, TN, jobs);
      }
      trsm_left_t_block(ctx, pb, L + p + (size_t)p * lda, lda, unit, nrhs, X + p, ldx);
    }
  }
}

// Linv = L^{-1} for an n x n lower-triangular L (unit diagonal if `unit`), Linv
// lower triangular (ld n).  Blocked substitution on the identity: row block p of
// Linv only has nonzeros in its first p + pb columns, so each step solves and
// updates only those (n^3/3 flops instead of n^3).
static void dense_trinv(tlr_ctx* ctx, int n, const double* L, int lda, int unit, double* Linv) {
  TLR_CUDA(cudaMemsetAsync(Linv, 0, sizeof(double) * (size_t)n * n, ctx->stream));
  add_diag(ctx, n, Linv, n, 1.0);
  for (int p = 0; p < n; p += NBK) {
    const int pb = std::min(NBK, n - p);
    trsm_left_block(ctx, pb, L + p + (size_t)p * lda, lda, unit, p + pb, Linv + p, n);
    const int m = n - p - pb;
    if (m > 0) {
      std::vector<GemmJob<double>> jobs{job<double>(NN, m, p + pb, L + (p + pb) + (size_t)p * lda, lda, Linv + p, n,
                                                    pb, Linv + p + pb, n, -1.0, 1.0)};
      gemm<double>(ctx, NN, jobs);
    }
  }
}

// ======================================================================== ARA engine
// Batched ARA (Algorithm 1) over `nops` operands T_op (n x n), with the dynamic
// batching of Algorithm 5: operands enter the batch in `order` (Algorithm 5
// sorts by original rank, descending), at most `max_slots` are sampled per
// round, converged operands leave the batch and the next ones take their
// place (updateSubset).  Gaussian blocks Omega_t (seed, stream, k, t) are
// shared by all operands in their t-th round.
struct Sampler {
  virtual ~Sampler() {}
  // Y[s] = T_{ops[s]} Omega for each slot s (Y[s] at Y + s*n*bs, leading dim n).
  virtual void sample(const std::vector<int>& ops, int t, const double* Om, double* Y) = 0;
  // B_op = T_op^T Q_op for every operand, given the final widths q.
  virtual void project(const std::vector<int>& q) = 0;
};

struct AraConfig {
  int n, bs;
  double eps;
  uint64_t seed;
  uint32_t stream, k;
  int max_slots;
};

struct AraStats {
  int64_t rounds = 0;     // sum over operands of their rounds
  int64_t batches = 0;    // number of batched rounds
  double flops = 0;       // orthogonalization flops (FP64)
};

static const double HALKO = 10.0 * sqrt(2.0 / M_PI);
static const double TAU_DROP = 1e-10;

// Q: nops x n x (n + bs) workspace; on return q[op] columns of Q_op are the basis.
static void ara_run(tlr_ctx* ctx, Sampler& S, int nops, const AraConfig& cf,
                    const std::vector<int>& order, double* Q, std::vector<int>& q, AraStats& st) {
  const int n = cf.n, bs = cf.bs;
  const size_t qstride = (size_t)n * (n + bs);
  const double thr = cf.eps / HALKO;
  q.assign(nops, 0);
  if (nops == 0) return;
  const int slots = std::max(1, std::min(cf.max_slots > 0 ? cf.max_slots : nops, nops));
  Buf bOm(ctx), bY(ctx), bW(ctx), bS(ctx), bG(ctx), bM(ctx), bSt(ctx), bE(ctx);
  double* Om = bOm.need<double>((size_t)n * bs);
  double* Y = bY.need<double>((size_t)slots * n * bs);
  double* W = bW.need<double>((size_t)slots * n * bs);
  double* Sb = bS.need<double>((size_t)slots * (n + bs) * bs);
  double* G = bG.need<double>((size_t)slots * bs * bs);
  double* M = bM.need<double>((size_t)slots * bs * bs);
  int* status = bSt.need<int>((size_t)slots * 2);
  double* en = bE.need<double>((size_t)slots);
  int* hs = static_cast<int*>(host_status(ctx, sizeof(int) * 2 * slots));

  std::vector<int> active;
  std::vector<int> round(nops, 0);
  size_t next = 0;
  auto refill = [&]() {
    while ((int)active.size() < slots && next < order.size()) active.push_back(order[next++]);
  };
  refill();
  int t_global = 0;
  while (!active.empty()) {
    const int ns = (int)active.size();
    // All slots of one batch share their round index only if they entered together;
    // Omega depends on the operand's own round, so group slots by round.
    std::vector<int> rounds_present;
    for (int op : active) rounds_present.push_back(round[op]);
    std::sort(rounds_present.begin(), rounds_present.end());
    rounds_present.erase(std::unique(rounds_present.begin(), rounds_present.end()), rounds_present.end());
    prof_mark(ctx, PH_SAMPLE);
    for (int t : rounds_present) {
      std::vector<int> ops_t, slot_t;
      for (int s = 0; s < ns; ++s)
        if (round[active[s]] == t) { ops_t.push_back(active[s]); slot_t.push_back(s); }
      omega(ctx, cf.seed, cf.stream, cf.k, (uint32_t)t, n, bs, Om);
      // sample into a contiguous staging area, then place at the slots' Y
      const bool contiguous = (slot_t.front() == 0 && slot_t.back() == (int)slot_t.size() - 1);
      if (contiguous) {
        S.sample(ops_t, t, Om, Y);
      } else {
        S.sample(ops_t, t, Om, W);
        std::vector<CopyJob> cj;
        for (size_t u = 0; u < slot_t.size(); ++u)
          cj.push_back(CopyJob{W + u * (size_t)n * bs, Y + (size_t)slot_t[u] * n * bs, (int64_t)n * bs});
        batched_copy(ctx, cj);
      }
    }
    // ---- orthog, iteration 1: Y <- Y - Q (Q^T Y); G = Y^T Y
    prof_mark(ctx, PH_ORTH);
    {
      std::vector<GemmJob<double>> j1, j2, j3;
      for (int s = 0; s < ns; ++s) {
        const int op = active[s];
        const double* Qo = Q + op * qstride;
        double* Ys = Y + (size_t)s * n * bs;
        double* Ss = Sb + (size_t)s * (n + bs) * bs;
        if (q[op] > 0) {
          j1.push_back(job<double>(TN, q[op], bs, Qo, n, Ys, n, n, Ss, q[op], 1.0, 0.0));
          j2.push_back(job<double>(NN, n, bs, Qo, n, Ss, q[op], q[op], Ys, n, -1.0, 1.0));
        }
        j3.push_back(job<double>(TN, bs, bs, Ys, n, Ys, n, n, G + (size_t)s * bs * bs, bs, 1.0, 0.0));
        st.flops += 4.0 * n * q[op] * bs + 2.0 * n * bs * bs;
      }
      gemm<double>(ctx, TN, j1);
      gemm<double>(ctx, NN, j2);
      gemm<double>(ctx, TN, j3);
      cholqr_small(ctx, ns, bs, G, M, status, en, thr, TAU_DROP, 1, nullptr);
      std::vector<GemmJob<double>> j4;
      for (int s = 0; s < ns; ++s)
        j4.push_back(job<double>(NN, n, bs, Y + (size_t)s * n * bs, n, M + (size_t)s * bs * bs, bs, bs,
                                 W + (size_t)s * n * bs, n, 1.0, 0.0));
      gemm<double>(ctx, NN, j4);
    }
    // ---- orthog, iteration 2 (re-orthogonalization): W <- W - Q (Q^T W); Cholesky-QR again
    {
      std::vector<GemmJob<double>> j1, j2, j3, j4;
      for (int s = 0; s < ns; ++s) {
        const int op = active[s];
        const double* Qo = Q + op * qstride;
        double* Ws = W + (size_t)s * n * bs;
        double* Ss = Sb + (size_t)s * (n + bs) * bs;
        if (q[op] > 0) {
          j1.push_back(job<double>(TN, q[op], bs, Qo, n, Ws, n, n, Ss, q[op], 1.0, 0.0));
          j2.push_back(job<double>(NN, n, bs, Qo, n, Ss, q[op], q[op], Ws, n, -1.0, 1.0));
        }
        j3.push_back(job<double>(TN, bs, bs, Ws, n, Ws, n, n, G + (size_t)s * bs * bs, bs, 1.0, 0.0));
        st.flops += 4.0 * n * q[op] * bs + 2.0 * n * bs * bs * 2;
      }
      gemm<double>(ctx, TN, j1);
      gemm<double>(ctx, NN, j2);
      gemm<double>(ctx, TN, j3);
      cholqr_small(ctx, ns, bs, G, M, status, en, thr, TAU_DROP, 0, status);
      for (int s = 0; s < ns; ++s) {
        const int op = active[s];
        j4.push_back(job<double>(NN, n, bs, W + (size_t)s * n * bs, n, M + (size_t)s * bs * bs, bs, bs,
                                 Q + op * qstride + (size_t)q[op] * n, n, 1.0, 0.0));
      }
      gemm<double>(ctx, NN, j4);
    }
    prof_mark(ctx, PH_SYNC);
    d2h_sync(ctx, hs, status, sizeof(int) * 2 * ns);
    st.batches++;
    std::vector<int> still;
    for (int s = 0; s < ns; ++s) {
      const int op = active[s];
      round[op]++;
      st.rounds++;
      const int conv = hs[2 * s], nk2 = hs[2 * s + 1];
      bool done = conv != 0;
      if (!done) {
        q[op] = std::min(q[op] + nk2, n);
        if (q[op] >= n || nk2 == 0) done = true;  // full basis, or no progress possible
      }
      if (!done && round[op] > 2 * n + 4) done = true;  // hard bound (each round adds >= 1 column)
      if (!done) still.push_back(op);
    }
    active.swap(still);
    refill();
    ++t_global;
  }
  prof_mark(ctx, PH_PROJECT);
  S.project(q);
}

// ---------------------------------------------------------------- dense operands
struct DenseSampler : Sampler {
  tlr_ctx* ctx;
  int n, bs;
  const double* T;  // nops x n x n
  const double* Q;
  size_t qstride;
  double* B;        // nops x n x n (first q columns used)
  double flops = 0;
  void sample(const std::vector<int>& ops, int, const double* Om, double* Y) override {
    std::vector<GemmJob<double>> jobs;
    for (size_t s = 0; s < ops.size(); ++s)
      jobs.push_back(job<double>(NN, n, bs, T + (size_t)ops[s] * n * n, n, Om, n, n, Y + s * (size_t)n * bs, n,
                                 1.0, 0.0));
    flops += 2.0 * n * n * bs * ops.size();
    gemm<double>(ctx, NN, jobs);
  }
  void project(const std::vector<int>& q) override {
    std::vector<GemmJob<double>> jobs;
    for (size_t op = 0; op < q.size(); ++op)
      if (q[op] > 0) {
        jobs.push_back(job<double>(TN, n, q[op], T + op * (size_t)n * n, n, Q + op * qstride, n, n,
                                   B + op * (size_t)n * n, n, 1.0, 0.0));
        flops += 2.0 * n * n * q[op];
      }
    gemm<double>(ctx, TN, jobs);
  }
};

}  // namespace tlr

// ======================================================================== TLR matrix helpers
static inline int64_t ix(const tlr_mat* M, int i, int j) { return (int64_t)i * M->nb + j; }
static inline double* Uptr(const tlr_mat* M, int i, int j) {
  return M->Urow[i] + (size_t)M->b * M->uoff[ix(M, i, j)];
}
static inline double* Vptr(const tlr_mat* M, int i, int j) {
  return M->Vcol[j] + (size_t)M->b * M->voff[ix(M, i, j)];
}

static void mat_free_storage(tlr_ctx* ctx, tlr_mat* M) {
  for (double* p : M->Urow) dfree(ctx, p);
  for (double* p : M->Vcol) dfree(ctx, p);
  M->Urow.assign(M->nb, nullptr);
  M->Vcol.assign(M->nb, nullptr);
}

static void mat_destroy(tlr_ctx* ctx, tlr_mat* M) {
  if (!M) return;
  mat_free_storage(ctx, M);
  dfree(ctx, M->pts);
  dfree(ctx, M->dperm);
  dfree(ctx, M->diag);
  dfree(ctx, M->dvec);
  dfree(ctx, M->dinv);
  delete M;
}

static tlr_mat* mat_new(int64_t N, int d, int b) {
  tlr_mat* M = new tlr_mat();
  M->N = N;
  M->d = d;
  M->b = b;
  M->nb = (int)std::max<int64_t>(1, (N + b - 1) / b);
  const int nb = M->nb;
  M->rank.assign((size_t)nb * nb, 0);
  M->uoff.assign((size_t)nb * nb, 0);
  M->voff.assign((size_t)nb * nb, 0);
  M->Urow.assign(nb, nullptr);
  M->Vcol.assign(nb, nullptr);
  M->ucap.assign(nb, 0);
  M->vlen.assign(nb, 0);
  M->ulen.assign(nb, 0);
  return M;
}

// ======================================================================== construction (tlr_compress)
// Points already in KD order on the device (pts_dev, N x d row-major); perm_host
// (may be null = identity) records the original index of each ordered point.
static void compress_ordered_impl(tlr_ctx* ctx, const double* pts_dev, const int64_t* perm_host, int64_t N, int d,
                                  const tlr_kernel* kern, int b, double eps, const tlr_opts* o, tlr_mat* M);

static void compress_impl(tlr_ctx* ctx, const double* pts_host, int64_t N, int d, const tlr_kernel* kern,
                          int b, double eps, const tlr_opts* o, tlr_mat* M) {
  std::vector<int64_t> perm(N);
  kd_order(pts_host, N, d, b, perm.data());
  std::vector<double> xo((size_t)N * d);
  for (int64_t p = 0; p < N; ++p)
    for (int q = 0; q < d; ++q) xo[p * d + q] = pts_host[perm[p] * d + q];
  Buf tmp(ctx);
  double* dp = tmp.need<double>((size_t)N * d);
  TLR_CUDA(cudaMemcpyAsync(dp, xo.data(), sizeof(double) * N * d, cudaMemcpyHostToDevice, ctx->stream));
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));  // xo is pageable and goes out of scope
  compress_ordered_impl(ctx, dp, perm.data(), N, d, kern, b, eps, o, M);
}

static void compress_ordered_impl(tlr_ctx* ctx, const double* pts_dev, const int64_t* perm_host, int64_t N, int d,
                                  const tlr_kernel* kern, int b, double eps, const tlr_opts* o, tlr_mat* M) {
  const int nb = M->nb;
  M->kern = *kern;
  M->eps = eps;
  M->perm.resize(N);
  for (int64_t p = 0; p < N; ++p) M->perm[p] = perm_host ? perm_host[p] : p;
  M->pts = static_cast<double*>(dalloc(ctx, sizeof(double) * std::max<int64_t>(1, N * d)));
  TLR_CUDA(cudaMemcpyAsync(M->pts, pts_dev, sizeof(double) * N * d, cudaMemcpyDeviceToDevice, ctx->stream));
  M->dperm = static_cast<int64_t*>(dalloc(ctx, sizeof(int64_t) * N));
  TLR_CUDA(cudaMemcpyAsync(M->dperm, M->perm.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, ctx->stream));
  M->diag = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b * b));
  {
    std::vector<int> ij;
    for (int k = 0; k < nb; ++k) { ij.push_back(k); ij.push_back(k); }
    const int* dij = static_cast<const int*>(upload(ctx, ij.data(), ij.size() * sizeof(int)));
    gen_tiles(ctx, M->pts, N, d, kern->ell, kern->nugget, b, dij, nb, M->diag);
  }
  // off-diagonal tiles, in batches
  std::vector<std::pair<int, int>> tiles;
  for (int j = 0; j < nb; ++j)
    for (int i = j + 1; i < nb; ++i) tiles.push_back({i, j});
  const int bs = o->bs;
  const size_t tile_bytes = sizeof(double) * (size_t)b * b;
  const int batch = (int)std::max<size_t>(1, std::min<size_t>(tiles.size(), (size_t)(3ull << 30) / (3 * tile_bytes)));
  Buf bT(ctx), bQ(ctx), bB(ctx);
  struct Stored { double* U; double* V; int r; };
  std::vector<Stored> st(tiles.size());
  std::vector<void*> chunks;
  for (size_t t0 = 0; t0 < tiles.size(); t0 += batch) {
    const int nt = (int)std::min<size_t>(batch, tiles.size() - t0);
    double* T = bT.need<double>((size_t)nt * b * b);
    double* Q = bQ.need<double>((size_t)nt * b * (b + bs));
    double* B = bB.need<double>((size_t)nt * b * b);
    std::vector<int> ij;
    for (int u = 0; u < nt; ++u) { ij.push_back(tiles[t0 + u].first); ij.push_back(tiles[t0 + u].second); }
    const int* dij = static_cast<const int*>(upload(ctx, ij.data(), ij.size() * sizeof(int)));
    gen_tiles(ctx, M->pts, N, d, kern->ell, kern->nugget, b, dij, nt, T);
    DenseSampler ds;
    ds.ctx = ctx; ds.n = b; ds.bs = bs; ds.T = T; ds.Q = Q; ds.qstride = (size_t)b * (b + bs); ds.B = B;
    AraConfig cf{b, bs, eps, o->seed, STREAM_COMPRESS, 0, 0};
    std::vector<int> order(nt);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int> q;
    AraStats as;
    ara_run(ctx, ds, nt, cf, order, Q, q, as);
    int64_t tot = 0;
    for (int u = 0; u < nt; ++u) tot += q[u];
    double* chunk = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(1, 2 * tot * b)));
    chunks.push_back(chunk);
    std::vector<CopyJob> cj;
    int64_t off = 0;
    for (int u = 0; u < nt; ++u) {
      Stored& s = st[t0 + u];
      s.r = q[u];
      s.U = chunk + off * b;
      s.V = chunk + (tot + off) * b;
      cj.push_back(CopyJob{Q + (size_t)u * b * (b + bs), s.U, (int64_t)q[u] * b});
      cj.push_back(CopyJob{B + (size_t)u * b * b, s.V, (int64_t)q[u] * b});
      off += q[u];
    }
    batched_copy(ctx, cj);
  }
  // panels: U in block rows, V in block columns
  for (size_t t = 0; t < tiles.size(); ++t) M->rank[ix(M, tiles[t].first, tiles[t].second)] = st[t].r;
  for (int i = 0; i < nb; ++i) {
    int64_t off = 0;
    for (int j = 0; j < i; ++j) { M->uoff[ix(M, i, j)] = off; off += M->rank[ix(M, i, j)]; }
    M->ulen[i] = off;
    M->ucap[i] = off;
    M->Urow[i] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(1, off) * b));
  }
  for (int j = 0; j < nb; ++j) {
    int64_t off = 0;
    for (int i = j + 1; i < nb; ++i) { M->voff[ix(M, i, j)] = off; off += M->rank[ix(M, i, j)]; }
    M->vlen[j] = off;
    M->Vcol[j] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(1, off) * b));
  }
  std::vector<CopyJob> cj;
  for (size_t t = 0; t < tiles.size(); ++t) {
    const int i = tiles[t].first, j = tiles[t].second;
    cj.push_back(CopyJob{st[t].U, Uptr(M, i, j), (int64_t)st[t].r * b});
    cj.push_back(CopyJob{st[t].V, Vptr(M, i, j), (int64_t)st[t].r * b});
  }
  batched_copy(ctx, cj);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  for (void* c : chunks) dfree(ctx, c);
  M->state = 0;
}

// ======================================================================== factorization
namespace tlr {

// Sampling chain of column k (Equation 2 / 3 regrouped with the Gram factors G_ij),
// evaluated in arithmetic T (double, or float for the mixed-precision path).  The
// ARA engine works in FP64: Omega arrives in FP64 and Y leaves in FP64; with
// T = float the chain's operands are FP32 copies of the panels and the products
// accumulate in FP32.
template <typename T>
struct FactorSampler : Sampler {
  tlr_ctx* ctx;
  const tlr_mat* A;  // input (compressed) matrix
  tlr_mat* F;        // factor under construction (columns < k final)
  const std::vector<T*>* FU;  // panels in arithmetic T (F->Urow, or FP32 copies)
  const std::vector<T*>* AU;  // A->Urow in T
  const std::vector<T*>* AV;  // A->Vcol in T
  int k, b, bs, Kk;
  const std::vector<int>* ops2i;  // operand -> tile row i
  BlkTables tb;
  const int64_t* goff_d;
  const int* gld_d;
  const T* Gbuf;
  T* X;              // Kk x bs
  T* X0;             // R0_k x bs
  Buf* wsamp;        // W blocks
  Buf* pbuf;
  Buf* zbuf;
  Buf* cbuf;         // FP32 staging (Omega, Y, Q, B) when T = float
  const double* Q;
  size_t qstride;
  double* Bcol;      // b x R_k (output of the projection, input of batchTrsm)
  std::vector<int64_t> boff;
  const std::vector<char>* member = nullptr;  // project only these operands (null: all)
  double flops_exec = 0, flops_model = 0;
  static constexpr bool F32 = sizeof(T) == 4;
  bool mine(int op) const { return !member || (*member)[op]; }

  const T* Uk(int i, int j) const { return (*FU)[i] + (size_t)b * F->uoff[ix(F, i, j)]; }
  const T* U0(int i) const { return (*AU)[i] + (size_t)b * A->uoff[ix(A, i, k)]; }
  const T* V0(int i) const { return (*AV)[k] + (size_t)b * A->voff[ix(A, i, k)]; }

  void sample(const std::vector<int>& ops, int, const double* Om64, double* Y64) override {
    const T* Om = reinterpret_cast<const T*>(Om64);
    T* Y = reinterpret_cast<T*>(Y64);
    if (F32) {
      float* st = cbuf->need<float>((size_t)b * bs * (1 + ops.size()));
      to_float(ctx, (int64_t)b * bs, Om64, st);
      Om = reinterpret_cast<const T*>(st);
      Y = reinterpret_cast<T*>(st + (size_t)b * bs);
    }
    // shared per round: X = Urow_k^T Omega, X0 = V0col_k^T Omega
    std::vector<GemmJob<T>> jx;
    const int64_t R0k = A->vlen[k];
    if (Kk > 0) jx.push_back(job<T>(TN, Kk, bs, (*FU)[k], b, Om, b, b, X, Kk, 1.0, 0.0));
    if (R0k > 0) jx.push_back(job<T>(TN, (int)R0k, bs, (*AV)[k], b, Om, b, b, X0, (int)R0k, 1.0, 0.0));
    gemm<T>(ctx, TN, jx);
    flops_exec += 2.0 * b * bs * (Kk + R0k);
    std::vector<SlotDesc> sd(ops.size());
    int64_t wtot = 0;
    for (size_t s = 0; s < ops.size(); ++s) {
      const int i = (*ops2i)[ops[s]];
      sd[s].i = i;
      sd[s].r0 = A->rank[ix(A, i, k)];
      sd[s].x0off = (int)A->voff[ix(A, i, k)];
      sd[s].Ki = (int)F->ulen[i];
      sd[s].woff = wtot;
      sd[s].poff = 0;
      sd[s].q = bs;
      wtot += (int64_t)(sd[s].r0 + sd[s].Ki) * bs;
    }
    T* W = wsamp->need<T>((size_t)wtot);
    const SlotDesc* sdd = static_cast<const SlotDesc*>(upload(ctx, sd.data(), sd.size() * sizeof(SlotDesc)));
    blkdiag_sample<T>(ctx, tb, (int)ops.size(), sdd, goff_d, gld_d, Gbuf, X, std::max(Kk, 1), X0,
                      (int)std::max<int64_t>(R0k, 1), bs, W);
    std::vector<GemmJob<T>> jy;
    for (size_t s = 0; s < ops.size(); ++s) {
      const int i = sd[s].i, r0 = sd[s].r0, Ki = sd[s].Ki;
      const int ldw = std::max(r0 + Ki, 1);
      GemmJob<T> g = job<T>(NN, b, bs, r0 ? U0(i) : nullptr, b, W + sd[s].woff, ldw, r0, Y + s * (size_t)b * bs, b,
                            1.0, 0.0);
      g.A[1] = (*FU)[i];
      g.lda[1] = b;
      g.B[1] = W + sd[s].woff + r0;
      g.ldb[1] = ldw;
      g.K[1] = Ki;
      jy.push_back(g);
      flops_exec += 2.0 * b * bs * (r0 + Ki);
      // paper model: 4 products per (i,j) pair, Equation 2
      double R = r0;
      for (int j = 0; j < k; ++j) R += F->rank[ix(F, i, j)] + F->rank[ix(F, k, j)];
      flops_model += 4.0 * b * bs * R;
    }
    gemm<T>(ctx, NN, jy);
    if (F32) to_double(ctx, (int64_t)b * bs * ops.size(), reinterpret_cast<const float*>(Y), Y64);
  }

  void project(const std::vector<int>& q) override {
    const int nops = (int)q.size();
    std::vector<SlotDesc> sd(nops);
    int64_t ptot = 0, ztot = 0, btot = 0;
    boff.assign(nops, 0);
    for (int op = 0; op < nops; ++op) {
      const int i = (*ops2i)[op];
      sd[op].i = i;
      sd[op].r0 = A->rank[ix(A, i, k)];
      sd[op].x0off = 0;
      sd[op].Ki = (int)F->ulen[i];
      sd[op].q = q[op];
      sd[op].poff = ptot;
      sd[op].woff = ztot;
      ptot += (int64_t)(sd[op].r0 + sd[op].Ki) * q[op];
      ztot += (int64_t)(sd[op].r0 + Kk) * q[op];
      boff[op] = btot;
      btot += q[op];
    }
    T* P = pbuf->need<T>((size_t)std::max<int64_t>(ptot, 1));
    T* Z = zbuf->need<T>((size_t)std::max<int64_t>(ztot, 1));
    // Q_i (and the output B) in arithmetic T
    const T* Qt = reinterpret_cast<const T*>(Q);
    size_t qs = qstride;
    T* Bt = reinterpret_cast<T*>(Bcol);
    if (F32) {
      float* st = cbuf->need<float>((size_t)2 * b * std::max<int64_t>(btot, 1));
      std::vector<ConvJob> cj;
      for (int op = 0; op < nops; ++op)
        if (mine(op)) cj.push_back(ConvJob{Q + op * qstride, st + (size_t)boff[op] * b, (int64_t)q[op] * b});
      batched_to_float(ctx, cj);
      Qt = reinterpret_cast<const T*>(st);
      qs = 0;  // per-op offsets come from boff below
      Bt = reinterpret_cast<T*>(st + (size_t)b * std::max<int64_t>(btot, 1));
    }
    auto Qop = [&](int op) -> const T* {
      return F32 ? Qt + (size_t)boff[op] * b : Qt + op * qs;
    };
    std::vector<GemmJob<T>> jp;
    for (int op = 0; op < nops; ++op) {
      if (q[op] == 0 || !mine(op)) continue;
      const int i = sd[op].i, r0 = sd[op].r0, Ki = sd[op].Ki;
      const int ldp = r0 + Ki;
      if (r0 > 0) jp.push_back(job<T>(TN, r0, q[op], U0(i), b, Qop(op), b, b, P + sd[op].poff, ldp, 1.0, 0.0));
      if (Ki > 0) jp.push_back(job<T>(TN, Ki, q[op], (*FU)[i], b, Qop(op), b, b, P + sd[op].poff + r0, ldp, 1.0, 0.0));
      flops_exec += 2.0 * b * q[op] * (r0 + Ki);
    }
    gemm<T>(ctx, TN, jp);
    const SlotDesc* sdd = static_cast<const SlotDesc*>(upload(ctx, sd.data(), sd.size() * sizeof(SlotDesc)));
    int qmax = 0;
    for (int v : q) qmax = std::max(qmax, v);
    blkdiag_project<T>(ctx, tb, nops, sdd, goff_d, gld_d, Gbuf, P, Z, Kk, qmax);
    std::vector<GemmJob<T>> jb;
    for (int op = 0; op < nops; ++op) {
      if (q[op] == 0 || !mine(op)) continue;
      const int i = sd[op].i, r0 = sd[op].r0;
      const int ldz = r0 + Kk;
      GemmJob<T> g = job<T>(NN, b, q[op], r0 ? V0(i) : nullptr, b, Z + sd[op].woff, std::max(ldz, 1), r0,
                            Bt + (size_t)boff[op] * b, b, 1.0, 0.0);
      g.A[1] = (*FU)[k];
      g.lda[1] = b;
      g.B[1] = Z + sd[op].woff + r0;
      g.ldb[1] = std::max(ldz, 1);
      g.K[1] = Kk;
      jb.push_back(g);
      flops_exec += 2.0 * b * q[op] * (r0 + Kk);
      double R = r0;
      for (int j = 0; j < k; ++j) R += F->rank[ix(F, i, j)] + F->rank[ix(F, k, j)];
      flops_model += 4.0 * b * q[op] * R;
    }
    gemm<T>(ctx, NN, jb);
    if (F32) {
      if (!member) {
        to_double(ctx, (int64_t)b * btot, reinterpret_cast<const float*>(Bt), Bcol);
      } else {
        for (int op = 0; op < nops; ++op)
          if (mine(op) && q[op])
            to_double(ctx, (int64_t)b * q[op], reinterpret_cast<const float*>(Bt) + (size_t)boff[op] * b,
                      Bcol + (size_t)boff[op] * b);
      }
    }
  }
};

// Per-tile precision rule: within one round, tiles whose estimated FP32 rounding
// error is far below the ARA threshold sample in FP32, the others in FP64.
struct MixedSampler : Sampler {
  tlr_ctx* ctx;
  int b, bs;
  FactorSampler<double>* f64;
  FactorSampler<float>* f32;
  std::vector<char> is32, is64;
  Buf* tmp;
  int64_t ops32 = 0, ops64 = 0;
  void sample(const std::vector<int>& ops, int t, const double* Om, double* Y) override {
    std::vector<int> o32, o64, s32, s64;
    for (size_t s = 0; s < ops.size(); ++s) {
      if (is32[ops[s]]) { o32.push_back(ops[s]); s32.push_back((int)s); }
      else { o64.push_back(ops[s]); s64.push_back((int)s); }
    }
    ops32 += (int64_t)o32.size();
    ops64 += (int64_t)o64.size();
    if (o64.empty()) { f32->sample(ops, t, Om, Y); return; }
    if (o32.empty()) { f64->sample(ops, t, Om, Y); return; }
    double* T = tmp->need<double>((size_t)b * bs * ops.size());
    f32->sample(o32, t, Om, T);
    f64->sample(o64, t, Om, T + (size_t)b * bs * o32.size());
    std::vector<CopyJob> cj;
    for (size_t u = 0; u < o32.size(); ++u)
      cj.push_back(CopyJob{T + u * (size_t)b * bs, Y + (size_t)s32[u] * b * bs, (int64_t)b * bs});
    for (size_t u = 0; u < o64.size(); ++u)
      cj.push_back(CopyJob{T + (o32.size() + u) * (size_t)b * bs, Y + (size_t)s64[u] * b * bs, (int64_t)b * bs});
    batched_copy(ctx, cj);
  }
  void project(const std::vector<int>& q) override {
    f32->member = &is32;
    f64->member = &is64;
    f32->project(q);
    f64->project(q);
  }
};

}  // namespace tlr

// Ensure Urow[i] of F has room for `extra` more columns (grow by copy).
static void ensure_ucap(tlr_ctx* ctx, tlr_mat* F, int i, int64_t extra) {
  const int b = F->b;
  if (F->ulen[i] + extra <= F->ucap[i] && F->Urow[i]) return;
  int64_t cap = std::max<int64_t>({F->ulen[i] + extra, F->ucap[i] * 3 / 2, 16});
  double* p = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)cap * b));
  if (F->ulen[i] > 0)
    TLR_CUDA(cudaMemcpyAsync(p, F->Urow[i], sizeof(double) * (size_t)F->ulen[i] * b, cudaMemcpyDeviceToDevice,
                             ctx->stream));
  dfree(ctx, F->Urow[i]);
  F->Urow[i] = p;
  F->ucap[i] = cap;
}

// Left-looking TLR Cholesky (Algorithm 6) / LDL^T (Algorithm 10).
// A is consumed; on success its storage is replaced by the factor.
static tlr_status factor_impl(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* o, int ldl) {
  const auto t_start = std::chrono::steady_clock::now();
  const int nb = A->nb, b = A->b, bs = o->bs;
  tlr_mat* F = mat_new(A->N, A->d, b);
  F->kern = A->kern;
  F->eps = eps;
  F->diag = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b * b));
  TLR_CUDA(cudaMemcpyAsync(F->diag, A->diag, sizeof(double) * (size_t)nb * b * b, cudaMemcpyDeviceToDevice,
                           ctx->stream));
  if (ldl) F->dvec = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b));
  F->dinv = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b * b));
  for (int i = 0; i < nb; ++i) ensure_ucap(ctx, F, i, std::max<int64_t>(A->ulen[i], 16));
  Buf bQ(ctx), bX(ctx), bX0(ctx), bG(ctx), bE(ctx), bW(ctx), bP(ctx), bZ(ctx), bTab(ctx), bInfo(ctx),
      bDV(ctx), bTmp(ctx), bDk(ctx), bBc(ctx);
  const size_t qstride = (size_t)b * (b + bs);
  double* Q = bQ.need<double>((size_t)std::max(nb - 1, 1) * qstride);
  int* info = bInfo.need<int>(2);
  bTmp.need<double>((size_t)b * NBK);  // sized once: the side stream never reallocates it
  double fl_exec = 0, fl_model = 0, fl_exec32 = 0;
  int64_t rounds = 0;
  std::vector<int> rtab((size_t)nb * nb * 3);
  // Mixed precision (precision policy): the sampling / projection chains run in FP32
  // on FP32 copies of the panels when eps >= 1e-4; everything else stays FP64.
  const bool mixed = o->precision == TLR_PREC_FP32 && eps >= 1e-4;
  std::vector<float*> AU32(nb, nullptr), AV32(nb, nullptr), FU32(nb, nullptr), FV32(nb, nullptr);
  std::vector<int64_t> fu32cap(nb, 0);
  Buf bG32(ctx), bX32(ctx), bX032(ctx), bDV32(ctx), bC32(ctx);
  auto f32_alloc = [&](int64_t n) { return static_cast<float*>(dalloc(ctx, sizeof(float) * (size_t)std::max<int64_t>(n, 1))); };
  if (mixed) {
    std::vector<ConvJob> cj;
    for (int i = 0; i < nb; ++i) {
      AU32[i] = f32_alloc((int64_t)b * A->ulen[i]);
      AV32[i] = f32_alloc((int64_t)b * A->vlen[i]);
      cj.push_back(ConvJob{A->Urow[i], AU32[i], (int64_t)b * A->ulen[i]});
      cj.push_back(ConvJob{A->Vcol[i], AV32[i], (int64_t)b * A->vlen[i]});
      fu32cap[i] = F->ucap[i];
      FU32[i] = f32_alloc((int64_t)b * fu32cap[i]);
    }
    batched_to_float(ctx, cj);
  }
  // Frobenius norms of the tiles (|A_ik|_F = |V0_ik|_F and |L_ij|_F = |V_ij|_F, U orthonormal)
  std::vector<double> nA((size_t)nb * nb, 0.0), nL((size_t)nb * nb, 0.0);
  Buf bNrm(ctx), bMix(ctx);
  int64_t tiles32 = 0, tiles64 = 0;
  auto panel_tile_norms = [&](const tlr_mat* M, int j, std::vector<double>& out) {
    const int64_t n = M->vlen[j];
    if (n == 0) return;
    double* d = bNrm.need<double>((size_t)n);
    col_sqnorms(ctx, M->Vcol[j], b, n, d);
    std::vector<double> h(n);
    TLR_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int i = j + 1; i < nb; ++i) {
      double sq = 0;
      for (int c = 0; c < M->rank[ix(M, i, j)]; ++c) sq += h[M->voff[ix(M, i, j)] + c];
      out[ix(M, i, j)] = std::sqrt(sq);
    }
  };
  if (mixed)
    for (int j = 0; j < nb; ++j) panel_tile_norms(A, j, nA);
  struct F32Guard {  // frees the FP32 copies on every exit path
    tlr_ctx* c;
    std::vector<float*>* v[4];
    ~F32Guard() {
      for (auto* vv : v)
        for (float* p : *vv) dfree(c, p);
    }
  } f32guard{ctx, {&AU32, &AV32, &FU32, &FV32}};

  for (int k = 0; k < nb; ++k) {
    const int Kk = (int)F->ulen[k];
    // ---- Gram factors of column k: Gcol_j = V(j)[i >= k]^T [D_j] V_kj, j < k
    prof_mark(ctx, PH_GRAM);
    std::vector<int64_t> goff(std::max(k, 1), 0);
    std::vector<int> gld(std::max(k, 1), 1);
    int64_t gtot = 0;
    for (int j = 0; j < k; ++j) {
      goff[j] = gtot;
      gld[j] = (int)std::max<int64_t>(1, F->vlen[j] - F->voff[ix(F, k, j)]);
      gtot += (int64_t)gld[j] * F->rank[ix(F, k, j)];
    }
    double* G = bG.need<double>((size_t)std::max<int64_t>(gtot, 1));
    float* G32 = mixed ? bG32.need<float>((size_t)std::max<int64_t>(gtot, 1)) : nullptr;
    {
      std::vector<GemmJob<double>> jg;
      std::vector<GemmJob<float>> jg32;
      std::vector<ConvJob> cdv;
      int64_t dvtot = 0;
      for (int j = 0; j < k; ++j) dvtot += (int64_t)b * F->rank[ix(F, k, j)];
      double* DV = ldl ? bDV.need<double>((size_t)std::max<int64_t>(dvtot, 1)) : nullptr;
      float* DV32 = (ldl && mixed) ? bDV32.need<float>((size_t)std::max<int64_t>(dvtot, 1)) : nullptr;
      int64_t dvo = 0;
      for (int j = 0; j < k; ++j) {
        const int rkj = F->rank[ix(F, k, j)];
        if (rkj == 0) continue;
        const int S = (int)(F->vlen[j] - F->voff[ix(F, k, j)]);
        const double* Vkj = Vptr(F, k, j);
        const float* Vkj32 = mixed ? FV32[j] + (size_t)b * F->voff[ix(F, k, j)] : nullptr;
        if (ldl) {  // D_j V_kj (Equation 3: D(j,j) inside the chain)
          scale_rows(ctx, b, rkj, F->dvec + (size_t)j * b, 0, Vkj, b, DV + dvo, b);
          Vkj = DV + dvo;
          if (mixed) {
            cdv.push_back(ConvJob{DV + dvo, DV32 + dvo, (int64_t)b * rkj});
            Vkj32 = DV32 + dvo;
          }
          dvo += (int64_t)b * rkj;
        }
        jg.push_back(job<double>(TN, S, rkj, Vptr(F, k, j), b, Vkj, b, b, G + goff[j], gld[j], 1.0, 0.0));
        fl_exec += 2.0 * b * S * rkj;
        if (mixed)  // FP32 Gram for the tiles that sample in FP32
          jg32.push_back(job<float>(TN, S, rkj, FV32[j] + (size_t)b * F->voff[ix(F, k, j)], b, Vkj32, b, b,
                                    G32 + goff[j], gld[j], 1.0, 0.0));
      }
      if (!cdv.empty()) batched_to_float(ctx, cdv);
      gemm<double>(ctx, TN, jg);
      gemm<float>(ctx, TN, jg32);
    }
    // The diagonal tile (updateDense, compensation, chol) is not read by the ARA of
    // column k, only by its batchTrsm: it runs on the side stream, overlapped with
    // the sampling rounds below, and is joined before the trsm.
    // (The Schur compensation runs a nested ARA with its own workspaces: it stays on the main stream.)
    const bool overlap = o->compensation != TLR_COMP_SCHUR;
    if (overlap) {
      TLR_CUDA(cudaEventRecord(ctx->ev_fork, ctx->main));
      TLR_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
      ctx->stream = ctx->side;
    }
    // ---- updateDense: A_kk -= sum_j U_kj G_kj U_kj^T  (G_kj = rows of tile k in Gcol_j)
    double* Akk = F->diag + (size_t)k * b * b;
    if (Kk > 0) {
      double* E = bE.need<double>((size_t)b * Kk);
      std::vector<GemmJob<double>> je;
      for (int j = 0; j < k; ++j) {
        const int rkj = F->rank[ix(F, k, j)];
        if (rkj == 0) continue;
        je.push_back(job<double>(NN, b, rkj, Uptr(F, k, j), b, G + goff[j], gld[j], rkj,
                                 E + (size_t)b * F->uoff[ix(F, k, j)], b, 1.0, 0.0));
        fl_exec += 2.0 * b * rkj * rkj;
      }
      gemm<double>(ctx, NN, je);
      const bool schur = (o->compensation == TLR_COMP_SCHUR);
      double* Dk = schur ? bDk.need<double>((size_t)b * b) : nullptr;
      std::vector<GemmJob<double>> jd{job<double>(NT, b, b, E, b, F->Urow[k], b, Kk, schur ? Dk : Akk, b,
                                                  schur ? 1.0 : -1.0, schur ? 0.0 : 1.0)};
      if (!schur) jd[0].flags = GEMM_TRIL;
      gemm<double>(ctx, NT, jd);
      fl_exec += (schur ? 2.0 : 1.0) * b * b * Kk;
      if (schur) {
        // Section 5.1.1: A_kk - D_k + diag(rowsum |D_k - Dbar_k|), Dbar_k = Q Q^T D_k Q Q^T,
        // Q from ARA of D_k to eps.
        axpy_matrix(ctx, b, b, -1.0, Dk, b, Akk, b);
        double* Id = bTmp.need<double>((size_t)b * b * 4 + (size_t)b * (b + bs));
        double* Qd = Id + (size_t)b * b;
        double* Bd = Qd + (size_t)b * (b + bs);
        DenseSampler ds;
        ds.ctx = ctx; ds.n = b; ds.bs = bs; ds.T = Dk; ds.Q = Qd; ds.qstride = (size_t)b * (b + bs); ds.B = Bd;
        AraConfig cf{b, bs, eps, o->seed, STREAM_SCHUR, (uint32_t)k, 1};
        std::vector<int> ord{0}, qd;
        AraStats as;
        ara_run(ctx, ds, 1, cf, ord, Qd, qd, as);
        const int r = qd[0];
        double* C1 = Bd + (size_t)b * b;        // Q^T D Q  (r x r)
        double* C2 = C1 + (size_t)b * b;        // Q C1     (b x r)
        // Bd = D^T Q = D Q (symmetric): C1 = Q^T Bd, C2 = Q C1, E = D - C2 Q^T
        if (r > 0) {
          std::vector<GemmJob<double>> a1{job<double>(TN, r, r, Qd, b, Bd, b, b, C1, r, 1.0, 0.0)};
          gemm<double>(ctx, TN, a1);
          std::vector<GemmJob<double>> a2{job<double>(NN, b, r, Qd, b, C1, r, r, C2, b, 1.0, 0.0)};
          gemm<double>(ctx, NN, a2);
          std::vector<GemmJob<double>> a3{job<double>(NT, b, b, C2, b, Qd, b, r, Dk, b, -1.0, 1.0)};
          gemm<double>(ctx, NT, a3);
        }
        add_rowsum_abs(ctx, b, Dk, b, Akk, b);
      }
    }
    if (o->compensation == TLR_COMP_SHIFT && o->shift != 0.0) add_diag(ctx, b, Akk, b, o->shift);
    // ---- dense factorization of the diagonal tile
    TLR_CUDA(cudaMemsetAsync(info, 0xff, sizeof(int), ctx->stream));
    dense_factor(ctx, b, Akk, b, ldl, ldl ? F->dvec + (size_t)k * b : nullptr, info, bTmp);
    fl_exec += (double)b * b * b / 3.0;
    fl_model += (double)b * b * b / 3.0;
    // L_kk^{-1}: batchTrsm becomes one product, and so does every later diagonal solve
    dense_trinv(ctx, b, Akk, b, ldl, F->dinv + (size_t)k * b * b);
    fl_exec += (double)b * b * b / 3.0;
    TLR_CUDA(cudaEventRecord(ctx->ev_join, ctx->stream));
    ctx->stream = ctx->main;
    auto check_tile = [&]() -> bool {
      TLR_CUDA(cudaStreamWaitEvent(ctx->main, ctx->ev_join, 0));
      int* hinfo = static_cast<int*>(host_status(ctx, 64));
      d2h_sync(ctx, hinfo, info, sizeof(int));
      return hinfo[0] < 0;
    };
    for (int j = 0; j < k; ++j) {
      const int r = F->rank[ix(F, k, j)];
      fl_model += 4.0 * b * r * r + 2.0 * b * b * r;
    }
    const int nops = nb - k - 1;
    if (nops == 0) {
      if (!check_tile()) {
        mat_destroy(ctx, F);
        A->state = 3;
        A->k_fail = k;
        return TLR_ERR_NOT_SPD;
      }
      continue;
    }
    // ---- cholARAUpdate (Algorithm 5): tiles sorted by their original rank, descending
    std::vector<int> ops2i(nops);
    for (int u = 0; u < nops; ++u) ops2i[u] = k + 1 + u;
    std::vector<int> order(nops);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
      return A->rank[ix(A, ops2i[a], k)] > A->rank[ix(A, ops2i[c], k)];
    });
    // device copies of the rank / offset tables
    for (int e = 0; e < nb * nb; ++e) {
      rtab[e] = F->rank[e];
      rtab[(size_t)nb * nb + e] = (int)F->uoff[e];
      rtab[(size_t)2 * nb * nb + e] = (int)F->voff[e];
    }
    int* dtab = bTab.need<int>((size_t)nb * nb * 3 + 2 * nb + 64);
    TLR_CUDA(cudaMemcpyAsync(dtab, rtab.data(), sizeof(int) * nb * nb * 3, cudaMemcpyHostToDevice, ctx->stream));
    int64_t* dgoff = reinterpret_cast<int64_t*>(dtab + (((size_t)nb * nb * 3 + 1) & ~size_t(1)));
    int* dgld = reinterpret_cast<int*>(dgoff + std::max(k, 1));
    TLR_CUDA(cudaMemcpyAsync(dgoff, goff.data(), sizeof(int64_t) * std::max(k, 1), cudaMemcpyHostToDevice, ctx->stream));
    TLR_CUDA(cudaMemcpyAsync(dgld, gld.data(), sizeof(int) * std::max(k, 1), cudaMemcpyHostToDevice, ctx->stream));
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));  // rtab / goff / gld are pageable
    FactorSampler<double> fs;
    FactorSampler<float> fs32;
    auto setup = [&](auto& f, auto* X, auto* X0, const void* Gb, auto* FUv, auto* AUv, auto* AVv) {
      f.ctx = ctx; f.A = A; f.F = F; f.k = k; f.b = b; f.bs = bs; f.Kk = Kk; f.ops2i = &ops2i;
      f.tb = BlkTables{dtab, dtab + (size_t)nb * nb, dtab + (size_t)2 * nb * nb, nb, k};
      f.goff_d = dgoff; f.gld_d = dgld;
      f.Gbuf = static_cast<decltype(f.Gbuf)>(Gb);
      f.X = X; f.X0 = X0;
      f.FU = FUv; f.AU = AUv; f.AV = AVv;
      f.wsamp = &bW; f.pbuf = &bP; f.zbuf = &bZ; f.cbuf = &bC32;
      f.Q = Q; f.qstride = qstride;
    };
    setup(fs, bX.need<double>((size_t)std::max(Kk, 1) * bs),
          bX0.need<double>((size_t)std::max<int64_t>(A->vlen[k], 1) * bs), G, &F->Urow, &A->Urow, &A->Vcol);
    MixedSampler ms;
    Sampler* smp = &fs;
    if (mixed) {
      setup(fs32, bX32.need<float>((size_t)std::max(Kk, 1) * bs),
            bX032.need<float>((size_t)std::max<int64_t>(A->vlen[k], 1) * bs), G32, &FU32, &AU32, &AV32);
      // estimated FP32 rounding error of tile i's chain: u32 sqrt(K) (|A_ik|_F + sum_j |L_ij|_F |L_kj|_F)
      const double thr = eps / HALKO;
      ms.ctx = ctx; ms.b = b; ms.bs = bs; ms.f64 = &fs; ms.f32 = &fs32; ms.tmp = &bMix;
      ms.is32.assign(nops, 0);
      ms.is64.assign(nops, 1);
      for (int op = 0; op < nops; ++op) {
        const int i = ops2i[op];
        double sum = nA[ix(A, i, k)];
        for (int j = 0; j < k; ++j) sum += nL[ix(F, i, j)] * nL[ix(F, k, j)];
        const double K = (double)A->rank[ix(A, i, k)] + (double)F->ulen[i] + bs;
        const bool ok = 6e-8 * std::sqrt(K) * sum <= thr / 8.0;
        ms.is32[op] = ok;
        ms.is64[op] = !ok;
      }
      smp = &ms;
    }
    // Bcol is allocated after ARA (R_k known) -> run ARA with a deferred projection
    struct Deferred : Sampler {
      Sampler* f;
      void sample(const std::vector<int>& ops, int t, const double* Om, double* Y) override { f->sample(ops, t, Om, Y); }
      void project(const std::vector<int>&) override {}
    } dsmp;
    dsmp.f = smp;
    AraConfig cf{b, bs, eps, o->seed, STREAM_FACTOR, (uint32_t)k, o->max_slots};
    std::vector<int> q;
    AraStats as;
    ara_run(ctx, dsmp, nops, cf, order, Q, q, as);
    rounds += as.rounds;
    fl_exec += as.flops;
    int64_t Rk = 0;
    for (int v : q) Rk += v;
    F->Vcol[k] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(Rk, 1) * b));
    F->vlen[k] = Rk;
    double* Bcol = bBc.need<double>((size_t)std::max<int64_t>(Rk, 1) * b);
    fs.Bcol = Bcol;
    fs32.Bcol = Bcol;
    prof_mark(ctx, PH_POTRF);  // waiting for the diagonal tile of this column
    if (!check_tile()) {
      mat_destroy(ctx, F);
      A->state = 3;
      A->k_fail = k;
      return TLR_ERR_NOT_SPD;
    }
    prof_mark(ctx, PH_PROJECT);
    smp->project(q);
    const std::vector<int64_t>& boff = fs.boff;
    fl_exec += fs.flops_exec;
    if (mixed) fl_exec32 += fs32.flops_exec;
    fl_model += fs.flops_model + (mixed ? fs32.flops_model : 0.0);
    if (mixed) { tiles32 += ms.ops32; tiles64 += ms.ops64; }
    // ---- batchTrsm: V_ik = L_kk^{-1} B_i (LDL^T: then D_k^{-1}, batchIDMult)
    prof_mark(ctx, PH_TRSM);
    if (Rk > 0) {
      std::vector<GemmJob<double>> jt{job<double>(NN, b, (int)Rk, F->dinv + (size_t)k * b * b, b, Bcol, b, b,
                                                  F->Vcol[k], b, 1.0, 0.0)};
      gemm<double>(ctx, NN, jt);
      if (ldl) scale_rows(ctx, b, (int)Rk, F->dvec + (size_t)k * b, 1, F->Vcol[k], b, F->Vcol[k], b);
      fl_exec += 2.0 * b * b * Rk;
      fl_model += (double)b * b * Rk;
    }
    // ---- updateTiles: U_ik = Q_i appended to block row i; V_ik in block column k
    prof_mark(ctx, PH_UPDATE);
    std::vector<CopyJob> cj;
    std::vector<ConvJob> c32;
    for (int op = 0; op < nops; ++op) {
      const int i = ops2i[op];
      ensure_ucap(ctx, F, i, q[op]);
      F->rank[ix(F, i, k)] = q[op];
      F->uoff[ix(F, i, k)] = F->ulen[i];
      F->voff[ix(F, i, k)] = boff[op];
      cj.push_back(CopyJob{Q + op * qstride, F->Urow[i] + (size_t)F->ulen[i] * b, (int64_t)q[op] * b});
      if (mixed) {
        if (F->ulen[i] + q[op] > fu32cap[i]) {  // grow the FP32 copy of block row i
          const int64_t cap = std::max<int64_t>(F->ucap[i], F->ulen[i] + q[op]);
          float* p = f32_alloc((int64_t)b * cap);
          if (F->ulen[i] > 0)
            TLR_CUDA(cudaMemcpyAsync(p, FU32[i], sizeof(float) * (size_t)b * F->ulen[i], cudaMemcpyDeviceToDevice,
                                     ctx->stream));
          dfree(ctx, FU32[i]);
          FU32[i] = p;
          fu32cap[i] = cap;
        }
        c32.push_back(ConvJob{Q + op * qstride, FU32[i] + (size_t)F->ulen[i] * b, (int64_t)q[op] * b});
      }
      F->ulen[i] += q[op];
    }
    batched_copy(ctx, cj);
    if (mixed) {
      FV32[k] = f32_alloc((int64_t)b * Rk);
      c32.push_back(ConvJob{F->Vcol[k], FV32[k], (int64_t)b * Rk});
      batched_to_float(ctx, c32);
      panel_tile_norms(F, k, nL);
    }
  }
  prof_flush(ctx);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  // A := F
  mat_free_storage(ctx, A);
  dfree(ctx, A->diag);
  dfree(ctx, A->dvec);
  A->diag = F->diag; F->diag = nullptr;
  A->dvec = F->dvec; F->dvec = nullptr;
  dfree(ctx, A->dinv);
  A->dinv = F->dinv; F->dinv = nullptr;
  A->rank = F->rank; A->uoff = F->uoff; A->voff = F->voff;
  A->Urow = F->Urow; A->Vcol = F->Vcol; A->ucap = F->ucap; A->vlen = F->vlen; A->ulen = F->ulen;
  F->Urow.assign(nb, nullptr);
  F->Vcol.assign(nb, nullptr);
  mat_destroy(ctx, F);
  A->state = ldl ? 2 : 1;
  A->k_fail = -1;
  A->eps = eps;
  A->flops_exec = fl_exec;
  A->flops_model = fl_model;
  A->ara_rounds = (double)rounds;
  A->tiles_fp32 = (double)tiles32;
  A->flops_fp32 = fl_exec32;
  A->tiles_fp64 = (double)tiles64;
  A->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return TLR_OK;
}

// ======================================================================== solve / products
// Z = L^{-1} X (Algorithm 7): Z_k = L_kk^{-1} X_k, then X_i -= U_ik (V_ik^T Z_k) for i > k.
// X (nb*b x nrhs, KD order, padded) is consumed.
static void tri_forward(tlr_ctx* ctx, const tlr_mat* F, int nrhs, double* X, double* Z, int64_t ld, Buf& tmp) {
  const int nb = F->nb, b = F->b;
  for (int k = 0; k < nb; ++k) {
    double* Zk = Z + (size_t)k * b;
    std::vector<GemmJob<double>> j0{job<double>(NN, b, nrhs, F->dinv + (size_t)k * b * b, b, X + (size_t)k * b, (int)ld,
                                                b, Zk, (int)ld, 1.0, 0.0)};
    gemm<double>(ctx, NN, j0);
    const int64_t Rk = F->vlen[k];
    if (Rk == 0) continue;
    double* T = tmp.need<double>((size_t)Rk * nrhs);
    std::vector<GemmJob<double>> j1{job<double>(TN, (int)Rk, nrhs, F->Vcol[k], b, Zk, (int)ld, b, T, (int)Rk, 1.0, 0.0)};
    gemm<double>(ctx, TN, j1);
    std::vector<GemmJob<double>> j2;
    for (int i = k + 1; i < nb; ++i) {
      const int r = F->rank[ix(F, i, k)];
      if (r == 0) continue;
      j2.push_back(job<double>(NN, b, nrhs, Uptr(F, i, k), b, T + F->voff[ix(F, i, k)], (int)Rk, r,
                               X + (size_t)i * b, (int)ld, -1.0, 1.0));
    }
    gemm<double>(ctx, NN, j2);
  }
}

// X = L^{-T} Z (transpose of Algorithm 7): Z_k -= sum_{i>k} V_ik (U_ik^T X_i); X_k = L_kk^{-T} Z_k.
static void tri_backward(tlr_ctx* ctx, const tlr_mat* F, int nrhs, double* Z, double* X, int64_t ld, Buf& tmp) {
  const int nb = F->nb, b = F->b;
  for (int k = nb - 1; k >= 0; --k) {
    double* Zk = Z + (size_t)k * b;
    const int64_t Rk = F->vlen[k];
    if (Rk > 0) {
      double* S = tmp.need<double>((size_t)Rk * nrhs);
      std::vector<GemmJob<double>> j1;
      for (int i = k + 1; i < nb; ++i) {
        const int r = F->rank[ix(F, i, k)];
        if (r == 0) continue;
        j1.push_back(job<double>(TN, r, nrhs, Uptr(F, i, k), b, X + (size_t)i * b, (int)ld, b,
                                 S + F->voff[ix(F, i, k)], (int)Rk, 1.0, 0.0));
      }
      gemm<double>(ctx, TN, j1);
      std::vector<GemmJob<double>> j2{job<double>(NN, b, nrhs, F->Vcol[k], b, S, (int)Rk, (int)Rk, Zk, (int)ld, -1.0, 1.0)};
      gemm<double>(ctx, NN, j2);
    }
    std::vector<GemmJob<double>> j3{job<double>(TN, b, nrhs, F->dinv + (size_t)k * b * b, b, Zk, (int)ld, b,
                                                X + (size_t)k * b, (int)ld, 1.0, 0.0)};
    gemm<double>(ctx, TN, j3);
  }
}

// Y = L X or Y = L^T X (KD order, padded); Y must not alias X.
static void tri_mul(tlr_ctx* ctx, const tlr_mat* F, int trans, int nrhs, const double* X, int64_t ldx, double* Y,
                    int64_t ldy, Buf& tmp) {
  const int nb = F->nb, b = F->b;
  const int unit = F->state == 2;
  // diagonal blocks: Y_k = L_kk X_k (or L_kk^T X_k) via the triangular tile as a dense GEMM on its lower part
  double* Lt = tmp.need<double>((size_t)b * b);
  for (int k = 0; k < nb; ++k) {
    // build a clean lower-triangular copy (unit diagonal for LDL^T)
    copy_matrix(ctx, b, b, F->diag + (size_t)k * b * b, b, Lt, b);
    std::vector<GemmJob<double>> jj;
    tril_mask(ctx, b, Lt, b, unit);
    jj.push_back(job<double>(trans ? TN : NN, b, nrhs, Lt, b, X + (size_t)k * b, (int)ldx, b, Y + (size_t)k * b,
                             (int)ldy, 1.0, 0.0));
    gemm<double>(ctx, trans ? TN : NN, jj);
  }
  Buf t2(ctx);
  for (int k = 0; k < nb; ++k) {
    const int64_t Rk = F->vlen[k];
    if (Rk == 0) continue;
    double* T = t2.need<double>((size_t)Rk * nrhs);
    if (!trans) {  // Y_i += U_ik (V_ik^T X_k)
      std::vector<GemmJob<double>> j1{job<double>(TN, (int)Rk, nrhs, F->Vcol[k], b, X + (size_t)k * b, (int)ldx, b, T,
                                                  (int)Rk, 1.0, 0.0)};
      gemm<double>(ctx, TN, j1);
      std::vector<GemmJob<double>> j2;
      for (int i = k + 1; i < nb; ++i) {
        const int r = F->rank[ix(F, i, k)];
        if (r) j2.push_back(job<double>(NN, b, nrhs, Uptr(F, i, k), b, T + F->voff[ix(F, i, k)], (int)Rk, r,
                                        Y + (size_t)i * b, (int)ldy, 1.0, 1.0));
      }
      gemm<double>(ctx, NN, j2);
    } else {  // Y_k += V_ik (U_ik^T X_i)
      std::vector<GemmJob<double>> j1;
      for (int i = k + 1; i < nb; ++i) {
        const int r = F->rank[ix(F, i, k)];
        if (r) j1.push_back(job<double>(TN, r, nrhs, Uptr(F, i, k), b, X + (size_t)i * b, (int)ldx, b,
                                        T + F->voff[ix(F, i, k)], (int)Rk, 1.0, 0.0));
      }
      gemm<double>(ctx, TN, j1);
      std::vector<GemmJob<double>> j2{job<double>(NN, b, nrhs, F->Vcol[k], b, T, (int)Rk, (int)Rk,
                                                  Y + (size_t)k * b, (int)ldy, 1.0, 1.0)};
      gemm<double>(ctx, NN, j2);
    }
  }
}

// Y = A X for the symmetric TLR matrix A (state 0), KD order, padded.
static void sym_mul(tlr_ctx* ctx, const tlr_mat* M, int nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  const int nb = M->nb, b = M->b;
  std::vector<GemmJob<double>> jd;
  for (int k = 0; k < nb; ++k)
    jd.push_back(job<double>(NN, b, nrhs, M->diag + (size_t)k * b * b, b, X + (size_t)k * b, (int)ldx, b,
                             Y + (size_t)k * b, (int)ldy, 1.0, 0.0));
  gemm<double>(ctx, NN, jd);
  Buf t(ctx), t2(ctx);
  for (int k = 0; k < nb; ++k) {
    const int64_t Rk = M->vlen[k];
    if (Rk == 0) continue;
    double* T = t.need<double>((size_t)Rk * nrhs);
    double* S = t2.need<double>((size_t)Rk * nrhs);
    std::vector<GemmJob<double>> j1{job<double>(TN, (int)Rk, nrhs, M->Vcol[k], b, X + (size_t)k * b, (int)ldx, b, T,
                                                (int)Rk, 1.0, 0.0)};
    gemm<double>(ctx, TN, j1);
    std::vector<GemmJob<double>> j2, j3;
    for (int i = k + 1; i < nb; ++i) {
      const int r = M->rank[ix(M, i, k)];
      if (!r) continue;
      j2.push_back(job<double>(NN, b, nrhs, Uptr(M, i, k), b, T + M->voff[ix(M, i, k)], (int)Rk, r, Y + (size_t)i * b,
                               (int)ldy, 1.0, 1.0));
      j3.push_back(job<double>(TN, r, nrhs, Uptr(M, i, k), b, X + (size_t)i * b, (int)ldx, b, S + M->voff[ix(M, i, k)],
                               (int)Rk, 1.0, 0.0));
    }
    gemm<double>(ctx, NN, j2);
    gemm<double>(ctx, TN, j3);
    std::vector<GemmJob<double>> j4{job<double>(NN, b, nrhs, M->Vcol[k], b, S, (int)Rk, (int)Rk, Y + (size_t)k * b,
                                                (int)ldy, 1.0, 1.0)};
    gemm<double>(ctx, NN, j4);
  }
}

// ======================================================================== C ABI
#define ABI_BEGIN try {
#define ABI_END                                     \
  }                                                 \
  catch (const tlr::Error& e) {                     \
    fprintf(stderr, "[tlr] %s\n", e.what());        \
    return e.status;                                \
  }                                                 \
  catch (const std::bad_alloc&) {                   \
    return TLR_ERR_NOMEM;                           \
  }                                                 \
  catch (...) {                                     \
    return TLR_ERR_CUDA;                            \
  }

extern "C" {

void tlr_opts_default(tlr_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->bs = 16;
  o->precision = TLR_PREC_FP64;
  o->compensation = TLR_COMP_NONE;
}

const char* tlr_strerror(tlr_status s) {
  switch (s) {
    case TLR_OK: return "ok";
    case TLR_ERR_ARG: return "invalid argument";
    case TLR_ERR_NOMEM: return "out of memory";
    case TLR_ERR_NOT_SPD: return "matrix not positive definite (tile factorization failed)";
    case TLR_ERR_CUDA: return "CUDA error";
    case TLR_ERR_TIMEOUT: return "device wait timed out";
    case TLR_ERR_STATE: return "object in the wrong state";
    case TLR_ERR_LIMIT: return "size above a compiled-in limit";
  }
  return "unknown status";
}

tlr_status tlr_create(tlr_ctx** out, int device, void* stream, tlr_alloc_fn alloc, tlr_free_fn free_fn, void* user) {
  if (!out || ((alloc == nullptr) != (free_fn == nullptr))) return TLR_ERR_ARG;
  tlr_ctx* ctx = nullptr;
  ABI_BEGIN
  ctx = new tlr_ctx();
  ctx->device = device;
  TLR_CUDA(cudaSetDevice(device));
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->main = ctx->stream;
  TLR_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  TLR_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  TLR_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  ctx->alloc = alloc;
  ctx->free_fn = free_fn;
  ctx->user = user;
  TLR_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
  ctx->ring_cap = 64ull << 20;
  TLR_CUDA(cudaMallocHost(&ctx->pinned, ctx->ring_cap));
  ctx->djobs = static_cast<char*>(dalloc(ctx, ctx->ring_cap));
  *out = ctx;
  return TLR_OK;
  }
  catch (const tlr::Error& e) {
    fprintf(stderr, "[tlr] %s\n", e.what());
    if (ctx) { if (ctx->pinned) cudaFreeHost(ctx->pinned); delete ctx; }
    return e.status;
  }
  catch (...) {
    if (ctx) delete ctx;
    return TLR_ERR_CUDA;
  }
}

tlr_status tlr_destroy(tlr_ctx* ctx) {
  if (!ctx) return TLR_ERR_ARG;
  ABI_BEGIN
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->side);
  dfree(ctx, ctx->djobs);
  dfree(ctx, ctx->scratch);
  dfree(ctx, ctx->scratch_side);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->hstatus) cudaFreeHost(ctx->hstatus);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (auto e : ctx->ev) cudaEventDestroy(e);
  for (auto e : ctx->kev) cudaEventDestroy(e);
  delete ctx;
  return TLR_OK;
  ABI_END
}

static tlr_opts opts_or_default(const tlr_opts* o) {
  tlr_opts r;
  if (o) r = *o; else tlr_opts_default(&r);
  if (r.bs <= 0) r.bs = 16;
  return r;
}

tlr_status tlr_compress(tlr_ctx* ctx, const double* pts, int64_t N, int d, const tlr_kernel* kern, int b,
                        double eps, const tlr_opts* opts, tlr_mat** A) {
  if (!ctx || !pts || !kern || !A || N <= 0 || d < 1 || d > 3 || b < 1 || !(eps > 0) || !(kern->ell > 0) ||
      kern->type != TLR_KERNEL_EXP || kern->nugget < 0)
    return TLR_ERR_ARG;
  tlr_opts o = opts_or_default(opts);
  if (o.bs > 64 || o.bs > b) return TLR_ERR_ARG;
  tlr_mat* M = nullptr;
  ABI_BEGIN
  M = mat_new(N, d, b);
  compress_impl(ctx, pts, N, d, kern, b, eps, &o, M);
  *A = M;
  return TLR_OK;
  }
  catch (const tlr::Error& e) {
    fprintf(stderr, "[tlr] %s\n", e.what());
    mat_destroy(ctx, M);
    return e.status;
  }
  catch (...) {
    return TLR_ERR_CUDA;
  }
}

tlr_status tlr_compress_ordered(tlr_ctx* ctx, const double* pts_dev, const int64_t* perm_host, int64_t N, int d,
                                const tlr_kernel* kern, int b, double eps, const tlr_opts* opts, tlr_mat** A) {
  if (!ctx || !pts_dev || !kern || !A || N <= 0 || d < 1 || d > 3 || b < 1 || !(eps > 0) || !(kern->ell > 0) ||
      kern->type != TLR_KERNEL_EXP || kern->nugget < 0)
    return TLR_ERR_ARG;
  tlr_opts o = opts_or_default(opts);
  if (o.bs > 64 || o.bs > b) return TLR_ERR_ARG;
  tlr_mat* M = nullptr;
  ABI_BEGIN
  M = mat_new(N, d, b);
  compress_ordered_impl(ctx, pts_dev, perm_host, N, d, kern, b, eps, &o, M);
  *A = M;
  return TLR_OK;
  }
  catch (const tlr::Error& e) {
    fprintf(stderr, "[tlr] %s\n", e.what());
    mat_destroy(ctx, M);
    return e.status;
  }
  catch (...) {
    return TLR_ERR_CUDA;
  }
}

tlr_status tlr_copy(tlr_ctx* ctx, const tlr_mat* S, tlr_mat** D) {
  if (!ctx || !S || !D) return TLR_ERR_ARG;
  ABI_BEGIN
  tlr_mat* M = new tlr_mat(*S);
  const int nb = S->nb, b = S->b;
  auto dup = [&](const double* src, size_t n) -> double* {
    if (!src) return nullptr;
    double* p = static_cast<double*>(dalloc(ctx, sizeof(double) * std::max<size_t>(n, 1)));
    if (n) TLR_CUDA(cudaMemcpyAsync(p, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return p;
  };
  M->pts = dup(S->pts, (size_t)S->N * S->d);
  M->dperm = reinterpret_cast<int64_t*>(dup(reinterpret_cast<const double*>(S->dperm), (size_t)S->N));
  M->diag = dup(S->diag, (size_t)nb * b * b);
  M->dvec = dup(S->dvec, (size_t)nb * b);
  M->dinv = dup(S->dinv, (size_t)nb * b * b);
  for (int i = 0; i < nb; ++i) {
    M->Urow[i] = S->Urow[i] ? dup(S->Urow[i], (size_t)std::max<int64_t>(S->ucap[i], 1) * b) : nullptr;
    M->Vcol[i] = S->Vcol[i] ? dup(S->Vcol[i], (size_t)std::max<int64_t>(S->vlen[i], 1) * b) : nullptr;
  }
  *D = M;
  return TLR_OK;
  ABI_END
}

static tlr_status factor_abi(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* opts, int ldl) {
  if (!ctx || !A || !(eps > 0)) return TLR_ERR_ARG;
  if (A->state != 0) return TLR_ERR_STATE;
  tlr_opts o = opts_or_default(opts);
  if (o.bs > 64 || o.bs > A->b || (o.precision != TLR_PREC_FP64 && o.precision != TLR_PREC_FP32)) return TLR_ERR_ARG;
  ABI_BEGIN
  return factor_impl(ctx, A, eps, &o, ldl);
  ABI_END
}

tlr_status tlr_potrf(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* o) { return factor_abi(ctx, A, eps, o, 0); }
tlr_status tlr_ldlt(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* o) { return factor_abi(ctx, A, eps, o, 1); }

tlr_status tlr_solve(tlr_ctx* ctx, const tlr_mat* F, int nrhs, double* B, int64_t ldb) {
  if (!ctx || !F || !B || nrhs < 0 || ldb < F->N) return TLR_ERR_ARG;
  if (F->state != 1 && F->state != 2) return TLR_ERR_STATE;
  if (nrhs == 0) return TLR_OK;
  ABI_BEGIN
  const int64_t np = (int64_t)F->nb * F->b;
  Buf bX(ctx), bZ(ctx), bT(ctx);
  double* X = bX.need<double>((size_t)np * nrhs);
  double* Z = bZ.need<double>((size_t)np * nrhs);
  const int64_t* perm = F->dperm;
  permute_rows(ctx, F->N, nrhs, perm, 1, B, ldb, X, np, np);
  tri_forward(ctx, F, nrhs, X, Z, np, bT);
  if (F->state == 2) scale_rows(ctx, (int)np, nrhs, F->dvec, 1, Z, (int)np, Z, (int)np);
  tri_backward(ctx, F, nrhs, Z, X, np, bT);
  permute_rows(ctx, F->N, nrhs, perm, 0, X, np, B, ldb, np);
  return TLR_OK;
  ABI_END
}

tlr_status tlr_logdet(tlr_ctx* ctx, const tlr_mat* F, double* logdet, int* sign) {
  if (!ctx || !F || !logdet) return TLR_ERR_ARG;
  if (F->state != 1 && F->state != 2) return TLR_ERR_STATE;
  ABI_BEGIN
  Buf b2(ctx);
  double* out = b2.need<double>(2);
  logdet_reduce(ctx, (int)F->N, F->diag, F->b, F->nb, F->state == 2 ? F->dvec : nullptr, out);
  double* h = static_cast<double*>(host_status(ctx, 64));
  d2h_sync(ctx, h, out, 2 * sizeof(double));
  *logdet = h[0];
  if (sign) *sign = (((int64_t)h[1]) % 2) ? -1 : 1;
  return TLR_OK;
  ABI_END
}

tlr_status tlr_matvec(tlr_ctx* ctx, const tlr_mat* F, int op, int nrhs, const double* X, int64_t ldx, double* Y,
                      int64_t ldy) {
  if (!ctx || !F || !X || !Y || nrhs < 0 || ldx < F->N || ldy < F->N) return TLR_ERR_ARG;
  if (op == TLR_OP_A ? F->state != 0 : (F->state != 1 && F->state != 2)) return TLR_ERR_STATE;
  if (op < 0 || op > 3) return TLR_ERR_ARG;
  if (nrhs == 0) return TLR_OK;
  ABI_BEGIN
  const int64_t np = (int64_t)F->nb * F->b;
  Buf bX(ctx), bY(ctx), bT(ctx), bZ(ctx);
  double* Xp = bX.need<double>((size_t)np * nrhs);
  double* Yp = bY.need<double>((size_t)np * nrhs);
  const int64_t* perm = F->dperm;
  permute_rows(ctx, F->N, nrhs, perm, 1, X, ldx, Xp, np, np);
  if (op == TLR_OP_A) sym_mul(ctx, F, nrhs, Xp, np, Yp, np);
  else if (op == TLR_OP_L) tri_mul(ctx, F, 0, nrhs, Xp, np, Yp, np, bT);
  else if (op == TLR_OP_LT) tri_mul(ctx, F, 1, nrhs, Xp, np, Yp, np, bT);
  else {
    double* Zp = bZ.need<double>((size_t)np * nrhs);
    tri_mul(ctx, F, 1, nrhs, Xp, np, Zp, np, bT);
    if (F->state == 2) scale_rows(ctx, (int)np, nrhs, F->dvec, 0, Zp, (int)np, Zp, (int)np);
    tri_mul(ctx, F, 0, nrhs, Zp, np, Yp, np, bT);
  }
  permute_rows(ctx, F->N, nrhs, perm, 0, Yp, np, Y, ldy, np);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_kernel_matvec(tlr_ctx* ctx, const double* pts, int64_t N, int d, const tlr_kernel* kern, int nrhs,
                             const double* X, int64_t ldx, double* Y, int64_t ldy) {
  if (!ctx || !pts || !kern || !X || !Y || N <= 0 || d < 1 || d > 3 || ldx < N || ldy < N || nrhs < 0 ||
      !(kern->ell > 0))
    return TLR_ERR_ARG;
  ABI_BEGIN
  Buf bp(ctx);
  double* dp = bp.need<double>((size_t)N * d);
  TLR_CUDA(cudaMemcpyAsync(dp, pts, sizeof(double) * N * d, cudaMemcpyHostToDevice, ctx->stream));
  kernel_matvec(ctx, dp, N, d, kern->ell, kern->nugget, nrhs, X, ldx, Y, ldy);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_get_info(const tlr_mat* M, tlr_info* info) {
  if (!M || !info) return TLR_ERR_ARG;
  memset(info, 0, sizeof(*info));
  info->N = M->N; info->b = M->b; info->nb = M->nb; info->d = M->d;
  info->state = M->state; info->k_fail = M->k_fail;
  int64_t sum = 0, cnt = 0;
  int mx = 0;
  for (int i = 0; i < M->nb; ++i)
    for (int j = 0; j < i; ++j) {
      const int r = M->rank[(size_t)i * M->nb + j];
      sum += r; ++cnt; mx = std::max(mx, r);
    }
  info->max_rank = mx;
  info->mean_rank = cnt ? (double)sum / cnt : 0.0;
  int64_t bytes = (int64_t)M->nb * M->b * M->b * 8 + (M->dvec ? (int64_t)M->nb * M->b * 8 : 0);
  bytes += 2 * sum * M->b * 8;
  info->bytes = bytes;
  info->flops_exec = M->flops_exec;
  info->flops_model = M->flops_model;
  info->ara_rounds = M->ara_rounds;
  info->seconds = M->seconds;
  info->flops_fp32 = M->flops_fp32;
  info->tile_rounds_fp32 = M->tiles_fp32;
  info->tile_rounds_fp64 = M->tiles_fp64;
  return TLR_OK;
}

tlr_status tlr_get_ranks(tlr_ctx*, const tlr_mat* M, int* ranks) {
  if (!M || !ranks) return TLR_ERR_ARG;
  for (size_t e = 0; e < M->rank.size(); ++e) ranks[e] = M->rank[e];
  return TLR_OK;
}

tlr_status tlr_get_perm(const tlr_mat* M, int64_t* perm) {
  if (!M || !perm) return TLR_ERR_ARG;
  for (int64_t p = 0; p < M->N; ++p) perm[p] = M->perm[p];
  return TLR_OK;
}

tlr_status tlr_get_tile(tlr_ctx* ctx, const tlr_mat* M, int i, int j, double* U, double* V) {
  if (!ctx || !M || i < 0 || j < 0 || i >= M->nb || j > i || !U) return TLR_ERR_ARG;
  ABI_BEGIN
  const int b = M->b;
  if (i == j) {
    TLR_CUDA(cudaMemcpyAsync(U, M->diag + (size_t)i * b * b, sizeof(double) * b * b, cudaMemcpyDeviceToHost, ctx->stream));
    if (V && M->dvec)
      TLR_CUDA(cudaMemcpyAsync(V, M->dvec + (size_t)i * b, sizeof(double) * b, cudaMemcpyDeviceToHost, ctx->stream));
  } else {
    const int r = M->rank[ix(M, i, j)];
    if (r) {
      TLR_CUDA(cudaMemcpyAsync(U, Uptr(M, i, j), sizeof(double) * b * r, cudaMemcpyDeviceToHost, ctx->stream));
      if (V) TLR_CUDA(cudaMemcpyAsync(V, Vptr(M, i, j), sizeof(double) * b * r, cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_free(tlr_ctx* ctx, tlr_mat* M) {
  if (!ctx || !M) return TLR_ERR_ARG;
  ABI_BEGIN
  mat_destroy(ctx, M);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_kd_order(const double* pts, int64_t N, int d, int b, int64_t* perm) {
  if (!pts || !perm || N < 0 || d < 1 || d > 3 || b < 1) return TLR_ERR_ARG;
  try {
    kd_order(pts, N, d, b, perm);
  } catch (...) {
    return TLR_ERR_NOMEM;
  }
  return TLR_OK;
}

tlr_status tlr_omega(tlr_ctx* ctx, uint64_t seed, uint32_t stream, uint32_t k, uint32_t t, int b, int bs, double* out) {
  if (!ctx || !out || b < 1 || bs < 1) return TLR_ERR_ARG;
  ABI_BEGIN
  omega(ctx, seed, stream, k, t, b, bs, out);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_ara_dense(tlr_ctx* ctx, int nops, int n, const double* T, int bs, double eps, uint64_t seed,
                         uint32_t stream, uint32_t k, double* Qout, double* Bout, int* rank) {
  if (!ctx || nops < 0 || n < 1 || !T || bs < 1 || bs > 64 || bs > n || !(eps > 0) || !Qout || !Bout || !rank)
    return TLR_ERR_ARG;
  if (nops == 0) return TLR_OK;
  ABI_BEGIN
  Buf bQ(ctx);
  const size_t qstride = (size_t)n * (n + bs);
  double* Q = bQ.need<double>((size_t)nops * qstride);
  DenseSampler ds;
  ds.ctx = ctx; ds.n = n; ds.bs = bs; ds.T = T; ds.Q = Q; ds.qstride = qstride; ds.B = Bout;
  AraConfig cf{n, bs, eps, seed, stream, k, 0};
  std::vector<int> order(nops), q;
  std::iota(order.begin(), order.end(), 0);
  AraStats as;
  ara_run(ctx, ds, nops, cf, order, Q, q, as);
  std::vector<CopyJob> cj;
  for (int op = 0; op < nops; ++op)
    cj.push_back(CopyJob{Q + op * qstride, Qout + (size_t)op * n * n, (int64_t)q[op] * n});
  batched_copy(ctx, cj);
  TLR_CUDA(cudaMemcpyAsync(rank, q.data(), sizeof(int) * nops, cudaMemcpyHostToDevice, ctx->stream));
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_dense_potrf(tlr_ctx* ctx, int n, double* A, int lda, int* info) {
  if (!ctx || !A || n < 0 || lda < n || !info) return TLR_ERR_ARG;
  ABI_BEGIN
  Buf bi(ctx), tmp(ctx);
  int* di = bi.need<int>(1);
  TLR_CUDA(cudaMemsetAsync(di, 0xff, sizeof(int), ctx->stream));
  dense_factor(ctx, n, A, lda, 0, nullptr, di, tmp);
  d2h_sync(ctx, info, di, sizeof(int));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_dense_ldlt(tlr_ctx* ctx, int n, double* A, int lda, int* info) {
  if (!ctx || !A || n < 0 || lda < n || !info) return TLR_ERR_ARG;
  ABI_BEGIN
  Buf bi(ctx), tmp(ctx), dv(ctx);
  int* di = bi.need<int>(1);
  double* d = dv.need<double>(std::max(n, 1));
  TLR_CUDA(cudaMemsetAsync(di, 0xff, sizeof(int), ctx->stream));
  dense_factor(ctx, n, A, lda, 1, d, di, tmp);
  // store D on the diagonal (unit L below it)
  set_diag(ctx, n, A, lda, d);
  d2h_sync(ctx, info, di, sizeof(int));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_dense_trsm(tlr_ctx* ctx, int n, const double* L, int lda, int unit, int nrhs, double* B, int ldb) {
  if (!ctx || !L || !B || n < 0 || lda < n || ldb < n || nrhs < 0) return TLR_ERR_ARG;
  ABI_BEGIN
  dense_trsm(ctx, n, L, lda, unit, nrhs, B, ldb, 0);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_fp64_peak(tlr_ctx* ctx, double* tflops) {
  if (!ctx || !tflops) return TLR_ERR_ARG;
  ABI_BEGIN
  *tflops = fp64_peak(ctx);
  return TLR_OK;
  ABI_END
}

int64_t tlr_launch_count(const tlr_ctx* ctx) { return ctx ? ctx->launches : -1; }

tlr_status tlr_gemm_stats(tlr_ctx* ctx, int enable, double* ms, double* flops, int64_t* launches) {
  if (!ctx) return TLR_ERR_ARG;
  ABI_BEGIN
  kprof_flush(ctx);
  for (int f = 0; f < 6; ++f) {
    if (ms) ms[f] = ctx->kfam_ms[f];
    if (flops) flops[f] = ctx->kfam_flops[f];
    if (launches) launches[f] = ctx->kfam_launches[f];
    ctx->kfam_ms[f] = 0; ctx->kfam_flops[f] = 0; ctx->kfam_launches[f] = 0;
  }
  ctx->kprof = enable != 0;
  return TLR_OK;
  ABI_END
}

tlr_status tlr_profile(tlr_ctx* ctx, int enable, double* ms, int64_t* launches, int n) {
  if (!ctx) return TLR_ERR_ARG;
  ABI_BEGIN
  prof_flush(ctx);
  if (ms)
    for (int p = 0; p < n && p < PH_COUNT; ++p) ms[p] = ctx->phase_ms[p];
  if (launches)
    for (int p = 0; p < n && p < PH_COUNT; ++p) launches[p] = ctx->phase_launch[p];
  if (ms && n > PH_COUNT) ms[PH_COUNT] = ctx->host_wait_ms;
  for (int p = 0; p < PH_COUNT; ++p) { ctx->phase_ms[p] = 0; ctx->phase_launch[p] = 0; }
  ctx->host_wait_ms = 0;
  ctx->prof = enable != 0;
  return TLR_OK;
  ABI_END
}

}  // extern "C"
