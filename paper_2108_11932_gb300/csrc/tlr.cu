// Host side of the GB300 TLR library: context and memory, the batched ARA
// engine with dynamic batching (Algorithm 1 + Algorithm 5), TLR construction,
// left-looking TLR Cholesky / LDL^T (Algorithm 6 / Algorithm 10), TLR solve
// (Algorithm 7), log-determinant, products, and the C ABI.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <cstdio>
#include <numeric>

#include "internal.h"

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
  ctx->live[p] = bytes;
  ctx->live_bytes += bytes;
  ctx->peak_bytes = std::max(ctx->peak_bytes, ctx->live_bytes);
  return p;
}

void dfree(tlr_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->live.find(p);
  if (it != ctx->live.end()) {
    ctx->live_bytes -= it->second;
    ctx->live.erase(it);
  }
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
int* split_counters(tlr_ctx* ctx, size_t n) {
  const int lane = (ctx->side && ctx->stream == ctx->side) ? 1 : 0;
  if (n > ctx->split_ctr_cap[lane]) {
    // earlier launches of this stream may still use the old array
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, ctx->split_ctr[lane]);
    ctx->split_ctr[lane] = nullptr;
    ctx->split_ctr_cap[lane] = 0;
    const size_t cap = std::max<size_t>(n, 1 << 16);
    ctx->split_ctr[lane] = static_cast<int*>(dalloc(ctx, cap * sizeof(int)));
    TLR_CUDA(cudaMemsetAsync(ctx->split_ctr[lane], 0, cap * sizeof(int), ctx->stream));
    ctx->split_ctr_cap[lane] = cap;
  }
  return ctx->split_ctr[lane];
}

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
    ctx->kev_bytes.resize(ctx->kev.size());
  }
  TLR_CUDA(cudaEventRecord(ctx->kev[ctx->kev_n], ctx->stream));
}

void kprof_end(tlr_ctx* ctx, int family, double flops, double bytes) {
  TLR_CUDA(cudaEventRecord(ctx->kev[ctx->kev_n + 1], ctx->stream));
  ctx->kev_fam[ctx->kev_n] = family;
  ctx->kev_flops[ctx->kev_n] = flops;
  ctx->kev_bytes[ctx->kev_n] = bytes;
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
    ctx->kfam_bytes[f] += ctx->kev_bytes[e];
    ctx->kfam_launches[f] += 1;
  }
  ctx->kev_n = 0;
}

void site_tick(tlr_ctx* ctx, const char* file, int line) { site_tick_on(ctx, ctx->stream, file, line); }

void site_tick_on(tlr_ctx* ctx, cudaStream_t stream, const char* file, int line) {
  const int lane = (ctx->side && stream == ctx->side) ? 1 : 0;
  if (!file) file = "gaps";
  const int phase = ctx->cur_phase < 0 ? 15 : ctx->cur_phase;  // phases < 16
  auto key = std::make_pair(file, (line * 2 + lane) * 16 + phase);
  auto it = ctx->site_id.find(key);
  int id;
  if (it == ctx->site_id.end()) {
    id = (int)ctx->site_name.size();
    const char* base = strrchr(file, '/');
    static const char* const pname[16] = {"gram", "diag_update", "potrf", "sample", "orthog", "host_sync",
                                          "project", "trsm", "update_tiles", "compress", "solve", "other",
                                          "p12", "p13", "p14", "-"};
    ctx->site_name.push_back(std::string(base ? base + 1 : file) + (line ? ":" + std::to_string(line) : std::string()) +
                             (lane ? "@side" : "@main") + "[" + pname[phase] + "]");
    ctx->site_ms.push_back(0.0);
    ctx->site_count.push_back(0);
    ctx->site_flops.push_back(0.0);
    ctx->site_id.emplace(key, id);
  } else {
    id = it->second;
  }
  auto& ev = ctx->sev[lane];
  size_t& n = ctx->sev_n[lane];
  if (n == ev.size()) {
    cudaEvent_t e;
    TLR_CUDA(cudaEventCreate(&e));
    ev.push_back(e);
    ctx->sev_site[lane].push_back(0);
    ctx->sev_flops[lane].push_back(0.0);
  }
  TLR_CUDA(cudaEventRecord(ev[n], stream));
  ctx->sev_site[lane][n] = id;
  ctx->sev_flops[lane][n] = file == std::string("gaps") ? 0.0 : ctx->site_next_flops;
  if (file != std::string("gaps")) ctx->site_next_flops = 0;
  ++n;
  if (n >= 8192) site_flush(ctx);
}

void site_flush(tlr_ctx* ctx) {
  TLR_CUDA(cudaStreamSynchronize(ctx->main));
  if (ctx->side) TLR_CUDA(cudaStreamSynchronize(ctx->side));
  for (int lane = 0; lane < 2; ++lane) {
    size_t& n = ctx->sev_n[lane];
    for (size_t e = 1; e < n; ++e) {
      float ms = 0;
      TLR_CUDA(cudaEventElapsedTime(&ms, ctx->sev[lane][e - 1], ctx->sev[lane][e]));
      ctx->site_ms[ctx->sev_site[lane][e]] += ms;
      ctx->site_count[ctx->sev_site[lane][e]] += 1;
      ctx->site_flops[ctx->sev_site[lane][e]] += ctx->sev_flops[lane][e];
    }
    if (n > 0) {  // the last event opens the next batch
      std::swap(ctx->sev[lane][0], ctx->sev[lane][n - 1]);
      ctx->sev_site[lane][0] = ctx->sev_site[lane][n - 1];
      ctx->sev_flops[lane][0] = ctx->sev_flops[lane][n - 1];
      n = 1;
    }
  }
}

void site_report(tlr_ctx* ctx) {
  if (!ctx->site_out) return;
  site_flush(ctx);
  std::vector<int> idx(ctx->site_name.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return ctx->site_ms[a] > ctx->site_ms[b]; });
  double tot = 0;
  for (double v : ctx->site_ms) tot += v;
  fprintf(ctx->site_out, "site\tlaunches\tms\tshare\tgflop\ttflops\n");
  for (int i : idx)
    if (ctx->site_count[i] > 0)
      fprintf(ctx->site_out, "%s\t%lld\t%.3f\t%.4f\t%.3f\t%.4f\n", ctx->site_name[i].c_str(),
              (long long)ctx->site_count[i], ctx->site_ms[i], tot > 0 ? ctx->site_ms[i] / tot : 0.0,
              ctx->site_flops[i] / 1e9, ctx->site_ms[i] > 0 ? ctx->site_flops[i] / ctx->site_ms[i] / 1e9 : 0.0);
  fflush(ctx->site_out);
}

void d2h_sync(tlr_ctx* ctx, void* host, const void* dev, size_t bytes) {
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
// Blocked right-looking Cholesky / unpivoted LDL^T of lower n x n tiles, all tiles
// of the batch advancing block by block in the same launches.  Each 64-column step:
// factor the diagonal block and invert its factor (one CTA per tile), apply the
// inverse to the panel below it (in place), and update the trailing lower triangle
// with one batched GEMM.  info (device int) must hold -1 on entry and receives the
// first failing column of its tile.  When a tile has Linv, the block inverses go to
// its diagonal blocks (dense_trinv_batch completes the inverse from them) and the
// rest of Linv is zeroed here; otherwise they go to tmp.
size_t dense_tmp_doubles(const std::vector<DenseTile>& tiles, int ldl) {
  size_t f = 0, t = 0;
  for (auto& x : tiles) {
    f += (ldl ? (size_t)x.n * NBK : 0) + (x.Linv ? 0 : (size_t)NBK * NBK);
    t += (size_t)x.n * x.n / 4 + NBK;
  }
  return std::max<size_t>(std::max(f, t), 1);
}

void dense_factor_batch(tlr_ctx* ctx, std::vector<DenseTile>& tiles, int ldl, Buf& tmp) {
  int nmax = 0;
  size_t wtot = 0;
  for (auto& t : tiles) {
    nmax = std::max(nmax, t.n);
    wtot += (ldl ? (size_t)t.n * NBK : 0) + (t.Linv ? 0 : (size_t)NBK * NBK);
    if (t.Linv) TLR_CUDA(cudaMemsetAsync(t.Linv, 0, sizeof(double) * (size_t)t.n * t.n, ctx->stream));
  }
  double* base = tmp.need<double>(std::max<size_t>(wtot, 1));
  std::vector<double*> Wt(tiles.size()), Bt(tiles.size());
  {
    size_t o = 0;
    for (size_t i = 0; i < tiles.size(); ++i) {
      Wt[i] = ldl ? base + o : nullptr;
      o += ldl ? (size_t)tiles[i].n * NBK : 0;
      Bt[i] = tiles[i].Linv ? nullptr : base + o;
      o += tiles[i].Linv ? 0 : (size_t)NBK * NBK;
    }
  }
  for (int p = 0; p < nmax; p += NBK) {
    std::vector<PotrfJob> pj;
    std::vector<PanelJob> qj;
    std::vector<GemmJob<double>> gj;
    for (size_t i = 0; i < tiles.size(); ++i) {
      auto& t = tiles[i];
      if (p >= t.n) continue;
      const int pb = std::min(NBK, t.n - p), lda = t.lda;
      double* App = t.A + p + (size_t)p * lda;
      double* Binv = t.Linv ? t.Linv + p + (size_t)p * t.n : Bt[i];
      const int ldb = t.Linv ? t.n : NBK;
      pj.push_back(PotrfJob{App, t.dvec, t.info, Binv, lda, p, pb, ldb});
      const int m = t.n - p - pb;
      if (m <= 0) continue;
      double* P = t.A + (p + pb) + (size_t)p * lda;
      qj.push_back(PanelJob{Binv, P, ldl ? t.dvec + p : nullptr, Wt[i], ldb, lda, m, pb});
      // trailing update: Cholesky P P^T; LDL^T W P^T with W = P D (written by the panel step)
      GemmJob<double> g = job<double>(NT, m, m, ldl ? Wt[i] : P, ldl ? m : lda, P, lda, pb,
                                      t.A + (p + pb) + (size_t)(p + pb) * lda, lda, -1.0, 1.0);
      g.flags = GEMM_TRIL;
      gj.push_back(g);
    }
    if (pj.empty()) break;
    potrf_inv_blocks(ctx, pj, ldl);
    panel_apply(ctx, qj, ldl);
    gemm<double>(ctx, NT, gj);
  }
}

// X = L^{-1} X (trans = 0) or X = L^{-T} X (trans = 1), L n x n lower.
void dense_trsm(tlr_ctx* ctx, int n, const double* L, int lda, int unit, int nrhs, double* X, int ldx, int trans) {
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

// Linv = L^{-1} for the tiles factored by dense_factor_batch (which left the
// inverses of the 64 x 64 diagonal blocks in Linv and zeros elsewhere).  Recursive
// doubling on the block lower-triangular structure: with Linv known on two
// consecutive diagonal blocks of width s, [A 0; B C]^{-1} = [A^-1 0; -C^-1 B A^-1 C^-1],
// so each level fills the off-diagonal blocks of all pairs with two batched GEMMs
// (T = B A^-1, then -C^-1 T).  log2(n / 64) levels; every level's products are
// large enough to occupy the whole GPU.
void dense_trinv_batch(tlr_ctx* ctx, std::vector<DenseTile>& tiles, int, Buf& tmp) {
  int nmax = 0;
  size_t ttot = 0;
  for (auto& t : tiles) {
    nmax = std::max(nmax, t.n);
    ttot += (size_t)t.n * t.n / 4 + NBK;
  }
  double* T = tmp.need<double>(std::max<size_t>(ttot, 1));
  for (int s = NBK; s < nmax; s *= 2) {
    std::vector<GemmJob<double>> j1, j2;
    size_t off = 0;
    for (auto& t : tiles) {
      const size_t tile_off = off;
      off += (size_t)t.n * t.n / 4 + NBK;
      size_t o2 = tile_off;
      for (int o = 0; o + s < t.n; o += 2 * s) {
        const int h = std::min(s, t.n - o - s);
        const double* B = t.A + (o + s) + (size_t)o * t.lda;
        const double* Ai = t.Linv + o + (size_t)o * t.n;
        const double* Ci = t.Linv + (o + s) + (size_t)(o + s) * t.n;
        double* Tp = T + o2;
        o2 += (size_t)h * s;
        j1.push_back(job<double>(NN, h, s, B, t.lda, Ai, t.n, s, Tp, h, 1.0, 0.0));
        j2.push_back(job<double>(NN, h, s, Ci, t.n, Tp, h, h, t.Linv + (o + s) + (size_t)o * t.n, t.n, -1.0, 0.0));
      }
    }
    gemm<double>(ctx, NN, j1);
    gemm<double>(ctx, NN, j2);
  }
}

// ======================================================================== ARA engine
// Batched ARA (Algorithm 1) over operands T_op (nrow[op] x nrow[op]), with the
// dynamic batching of Algorithm 5: operands enter the batch in `order`, at most
// `max_slots` are sampled per round, converged operands leave the batch and the
// next ones take their place (updateSubset).  Gaussian blocks: either drawn here,
// Omega_t (seed, stream, k, t) shared by all operands in their t-th round, or drawn
// by the sampler (one per matrix of a multi-matrix batch).
const double HALKO = 10.0 * sqrt(2.0 / M_PI);
const double TAU_DROP = 1e-10;

void ara_run(tlr_ctx* ctx, Sampler& S, const std::vector<int>& nrow, const std::vector<double>& thr,
             const AraConfig& cf, const std::vector<int>& order, double* Q, const std::vector<int64_t>& qoff,
             std::vector<int>& q, AraStats& st) {
  const int nops = (int)nrow.size(), bs = cf.bs;
  q.assign(nops, 0);
  if (nops == 0) return;
  int nmax = 0;
  for (int v : nrow) nmax = std::max(nmax, v);
  const int slots = std::max(1, std::min(cf.max_slots > 0 ? cf.max_slots : nops, nops));
  Buf bOm(ctx), bY(ctx), bW(ctx), bS(ctx), bG(ctx), bM(ctx), bSt(ctx), bE(ctx), bT(ctx), bOr(ctx);
  double* Om = S.owns_omega() ? nullptr : bOm.need<double>((size_t)nmax * bs);
  double* Y = bY.need<double>((size_t)slots * nmax * bs);
  double* W = bW.need<double>((size_t)slots * nmax * bs);
  double* Sb = bS.need<double>((size_t)slots * (nmax + bs) * bs);
  double* G = bG.need<double>((size_t)slots * bs * bs);
  double* M = bM.need<double>((size_t)slots * bs * bs);
  int* status = bSt.need<int>((size_t)slots * 2);
  double* en = bE.need<double>((size_t)slots);
  double* thr_d = bT.need<double>((size_t)slots);
  std::vector<double> thr_h(slots);

  std::vector<int> active;
  std::vector<int> round(nops, 0);
  bool any_fused = false;
  size_t next = 0;
  auto refill = [&]() {
    while ((int)active.size() < slots && next < order.size()) active.push_back(order[next++]);
  };
  refill();
  while (!active.empty()) {
    const int ns = (int)active.size();
    prof_mark(ctx, PH_SAMPLE);
    // Omega depends on the operand's own round: group the slots by round
    std::vector<int> rounds_present;
    for (int op : active) rounds_present.push_back(round[op]);
    std::sort(rounds_present.begin(), rounds_present.end());
    rounds_present.erase(std::unique(rounds_present.begin(), rounds_present.end()), rounds_present.end());
    for (int t : rounds_present) {
      std::vector<int> ops_t;
      std::vector<double*> ydst;
      for (int s = 0; s < ns; ++s)
        if (round[active[s]] == t) {
          ops_t.push_back(active[s]);
          ydst.push_back(Y + (size_t)s * nmax * bs);
        }
      if (Om) omega(ctx, cf.seed, cf.stream, cf.k, (uint32_t)t, nrow[ops_t[0]], bs, Om);
      S.sample(ops_t, t, Om, ydst);
    }
    prof_mark(ctx, PH_ORTH);
    bool fused = orth_fused_ok(bs);
    if (fused && !cf.fused_all) {
      double fma = 0;
      for (int s = 0; s < ns; ++s) fma += 4.0 * nrow[active[s]] * (double)bs * (q[active[s]] + bs);
      fused = fma <= ORTH_FUSED_MAX_FMA;
    }
    any_fused |= fused;
    if (fused) {  // both iterations below in one launch (k_orth.cu)
      std::vector<OrthSlot> os(ns);
      for (int s = 0; s < ns; ++s) {
        const int op = active[s], n = nrow[op];
        os[s] = OrthSlot{Q + qoff[op], Y + (size_t)s * nmax * bs, W + (size_t)s * nmax * bs, n, q[op], thr[op]};
        st.flops += 8.0 * n * q[op] * bs + 6.0 * n * bs * bs;
      }
      orth_round(ctx, bs, os, status, en, TAU_DROP, bOr);
    } else {
    for (int s = 0; s < ns; ++s) thr_h[s] = thr[active[s]];
    TLR_CUDA(cudaMemcpyAsync(thr_d, upload(ctx, thr_h.data(), sizeof(double) * ns), sizeof(double) * ns,
                             cudaMemcpyDeviceToDevice, ctx->stream));
    // ---- orthog, iteration 1: Y <- Y - Q (Q^T Y); G = Y^T Y
    {
      std::vector<GemmJob<double>> j1, j2, j3;
      for (int s = 0; s < ns; ++s) {
        const int op = active[s], n = nrow[op];
        const double* Qo = Q + qoff[op];
        double* Ys = Y + (size_t)s * nmax * bs;
        double* Ss = Sb + (size_t)s * (nmax + bs) * bs;
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
      cholqr_small(ctx, ns, bs, G, M, status, en, thr_d, TAU_DROP, 1, nullptr);
      std::vector<GemmJob<double>> j4;
      for (int s = 0; s < ns; ++s) {
        const int n = nrow[active[s]];
        j4.push_back(job<double>(NN, n, bs, Y + (size_t)s * nmax * bs, n, M + (size_t)s * bs * bs, bs, bs,
                                 W + (size_t)s * nmax * bs, n, 1.0, 0.0));
      }
      gemm<double>(ctx, NN, j4);
    }
    // ---- orthog, iteration 2 (re-orthogonalization): W <- W - Q (Q^T W); Cholesky-QR again
    {
      std::vector<GemmJob<double>> j1, j2, j3, j4;
      for (int s = 0; s < ns; ++s) {
        const int op = active[s], n = nrow[op];
        const double* Qo = Q + qoff[op];
        double* Ws = W + (size_t)s * nmax * bs;
        double* Ss = Sb + (size_t)s * (nmax + bs) * bs;
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
      cholqr_small(ctx, ns, bs, G, M, status, en, thr_d, TAU_DROP, 0, status);
      for (int s = 0; s < ns; ++s) {
        const int op = active[s], n = nrow[op];
        j4.push_back(job<double>(NN, n, bs, W + (size_t)s * nmax * bs, n, M + (size_t)s * bs * bs, bs, bs,
                                 Q + qoff[op] + (size_t)q[op] * n, n, 1.0, 0.0));
      }
      gemm<double>(ctx, NN, j4);
    }
    }
    prof_mark(ctx, PH_SYNC);
    int* hs = static_cast<int*>(host_status(ctx, sizeof(int) * 2 * slots));
    d2h_sync(ctx, hs, status, sizeof(int) * 2 * ns);
    st.batches++;
    std::vector<int> still;
    for (int s = 0; s < ns; ++s) {
      const int op = active[s], n = nrow[op];
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
  }
  if (any_fused)
    TLR_REQUIRE(!orth_timeout_flag(ctx), TLR_ERR_TIMEOUT, "orthogonalization: a bounded device wait ran out");
  prof_mark(ctx, PH_PROJECT);
  S.project(q);
}

// ---------------------------------------------------------------- dense operands
// With chunk planes (construction tiles: `oz`), both products run on the tensor cores by exact
// splitting (k_ozaki.cu): T Omega reads the row-oriented slices, T^T Q the column-oriented ones.
struct DenseSampler : Sampler {
  tlr_ctx* ctx;
  int n, bs;
  const double* T;  // nops x n x n
  const double* Q;
  const std::vector<int64_t>* qoff;
  double* B;        // nops x n x n (first q columns used)
  const OzTiles* oz = nullptr;
  double flops = 0;
  void sample(const std::vector<int>& ops, int, const double* Om, const std::vector<double*>& Ydst) override {
    flops += 2.0 * n * n * bs * ops.size();
    if (oz) {
      int8_t* Xs = oz->bx->need<int8_t>((size_t)8 * n * bs);
      int* ex = oz->be->need<int>((size_t)bs);
      std::vector<OzColJob> cj{OzColJob{Om, Xs, ex, n, bs, 0, n}};
      oz_split_cols(ctx, cj);
      std::vector<OzJob> jobs;
      for (size_t s = 0; s < ops.size(); ++s) {
        jobs.push_back(OzJob{oz->Sr + (size_t)ops[s] * 8 * n * n, Xs, oz->e + ops[s], ex, Ydst[s], (size_t)n * n,
                             (size_t)n * bs, n, n, n, bs, n});
        jobs.back().nsplit = 1;  // a batch of tiles fills the GPU without splitting K
        jobs.back().tol = oz->thr8 / std::sqrt((double)n);  // column norm of the sample within thr / 8
      }
      oz_gemm(ctx, jobs);
      return;
    }
    std::vector<GemmJob<double>> jobs;
    for (size_t s = 0; s < ops.size(); ++s)
      jobs.push_back(job<double>(NN, n, bs, T + (size_t)ops[s] * n * n, n, Om, n, n, Ydst[s], n, 1.0, 0.0));
    gemm<double>(ctx, NN, jobs);
  }
  void project(const std::vector<int>& q) override {
    for (size_t op = 0; op < q.size(); ++op) flops += 2.0 * n * n * q[op];
    if (oz) {
      int64_t cols = 0;
      for (int v : q) cols += v;
      if (cols == 0) return;
      int8_t* Xs = oz->bx->need<int8_t>((size_t)8 * n * cols);
      int* ex = oz->be->need<int>((size_t)cols);
      std::vector<OzColJob> cj;
      std::vector<OzJob> jobs;
      int64_t c0 = 0;
      for (size_t op = 0; op < q.size(); ++op) {
        if (q[op] == 0) continue;
        int8_t* xo = Xs + (size_t)8 * n * c0;
        cj.push_back(OzColJob{Q + (*qoff)[op], xo, ex + c0, n, q[op], 0, n});
        jobs.push_back(OzJob{oz->Sc + op * (size_t)8 * n * n, xo, oz->e + op, ex + c0, B + op * (size_t)n * n,
                             (size_t)n * n, (size_t)n * q[op], n, n, n, q[op], n});
        jobs.back().nsplit = 1;
        jobs.back().tol = oz->thr8 / std::sqrt((double)n * q[op]);  // Frobenius norm of B within thr / 8
        c0 += q[op];
      }
      oz_split_cols(ctx, cj);
      oz_gemm(ctx, jobs);
      return;
    }
    std::vector<GemmJob<double>> jobs;
    for (size_t op = 0; op < q.size(); ++op)
      if (q[op] > 0)
        jobs.push_back(job<double>(TN, n, q[op], T + op * (size_t)n * n, n, Q + (*qoff)[op], n, n,
                                   B + op * (size_t)n * n, n, 1.0, 0.0));
    gemm<double>(ctx, TN, jobs);
  }
};

// Uniform dense ARA (construction tiles, tlr_ara_dense, Schur compensation).
void ara_dense_run(tlr_ctx* ctx, int nops, int n, const double* T, int bs, double eps, uint64_t seed, uint32_t stream,
                   uint32_t k, double* Q, double* B, std::vector<int>& q, AraStats& st, const OzTiles* oz) {
  std::vector<int> nrow(nops, n), order(nops);
  std::vector<double> thr(nops, eps / HALKO);
  std::vector<int64_t> qoff(nops);
  for (int op = 0; op < nops; ++op) qoff[op] = (int64_t)op * n * (n + bs);
  std::iota(order.begin(), order.end(), 0);
  DenseSampler ds;
  ds.ctx = ctx; ds.n = n; ds.bs = bs; ds.T = T; ds.Q = Q; ds.qoff = &qoff; ds.B = B; ds.oz = oz;
  AraConfig cf{bs, seed, stream, k, 0};
  ara_run(ctx, ds, nrow, thr, cf, order, Q, qoff, q, st);
}

}  // namespace tlr

// ======================================================================== TLR matrix helpers
namespace tlr {

void mat_free_storage(tlr_ctx* ctx, tlr_mat* M) {
  mat_drop_plans(ctx, M);  // the plans point into the storage
  for (double* p : M->Urow) dfree(ctx, p);
  for (double* p : M->Vcol) dfree(ctx, p);
  M->Urow.assign(M->nb, nullptr);
  M->Vcol.assign(M->nb, nullptr);
}

void mat_destroy(tlr_ctx* ctx, tlr_mat* M) {
  if (!M) return;
  mat_free_storage(ctx, M);
  dfree(ctx, M->pts);
  dfree(ctx, M->dperm);
  dfree(ctx, M->diag);
  dfree(ctx, M->dvec);
  dfree(ctx, M->dinv);
  delete M;
}

tlr_mat* mat_new(int64_t N, int d, int b) {
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

}  // namespace tlr

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
  Buf bGx(ctx), bGi(ctx);
  long long* gx = bGx.need<long long>((size_t)N * d);
  GridInfo* ginfo = reinterpret_cast<GridInfo*>(bGi.need<double>(sizeof(GridInfo) / sizeof(double) + 1));
  grid_points(ctx, M->pts, N, d, ginfo, gx);
  {
    std::vector<int> ij;
    for (int k = 0; k < nb; ++k) { ij.push_back(k); ij.push_back(k); }
    const int* dij = static_cast<const int*>(upload(ctx, ij.data(), ij.size() * sizeof(int)));
    gen_tiles(ctx, gx, ginfo, N, d, kern->ell, kern->nugget, b, dij, nb, M->diag);
  }
  // Off-diagonal tiles, in batches of similar rank.  In KD order a tile's rank falls with its
  // distance from the diagonal, so the tiles are taken by diagonal offset i - j: a batch then
  // converges in about the same number of ARA rounds instead of waiting, round after round, for
  // its one near-diagonal tile.  Each tile's ARA is independent of its batch, so the order does
  // not change any result.
  std::vector<std::pair<int, int>> tiles;
  for (int off = 1; off < nb; ++off)
    for (int j = 0; j + off < nb; ++j) tiles.push_back({j + off, j});
  const int bs = o->bs;
  const size_t tile_bytes = sizeof(double) * (size_t)b * b;
  const int batch = (int)std::max<size_t>(1, std::min<size_t>(tiles.size(), (size_t)(3ull << 30) / (3 * tile_bytes)));
  Buf bT(ctx), bQ(ctx), bB(ctx), bMax(ctx), bSc(ctx), bSr(ctx), bEt(ctx), bXs(ctx), bEx(ctx);
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
    std::vector<int> q;
    AraStats as;
    if (b % 16 == 0) {  // the tensor-core split products read 16-byte rows of int8 chunks
      unsigned long long* tmax = bMax.need<unsigned long long>((size_t)nt);
      TLR_CUDA(cudaMemsetAsync(tmax, 0, sizeof(unsigned long long) * nt, ctx->stream));
      gen_tiles(ctx, gx, ginfo, N, d, kern->ell, kern->nugget, b, dij, nt, T, tmax);
      OzTiles oz;
      oz.Sc = bSc.need<int8_t>((size_t)nt * 8 * b * b);
      oz.Sr = bSr.need<int8_t>((size_t)nt * 8 * b * b);
      oz.e = bEt.need<int>((size_t)nt);
      oz.bx = &bXs;
      oz.be = &bEx;
      if (o->precision == TLR_PREC_MIXED && eps >= 1e-4) oz.thr8 = eps / HALKO / 8.0;
      oz_split_tiles(ctx, nt, b, T, tmax, oz.Sc, oz.Sr, oz.e);
      ara_dense_run(ctx, nt, b, T, bs, eps, o->seed, STREAM_COMPRESS, 0, Q, B, q, as, &oz);
    } else {
      gen_tiles(ctx, gx, ginfo, N, d, kern->ell, kern->nugget, b, dij, nt, T);
      ara_dense_run(ctx, nt, b, T, bs, eps, o->seed, STREAM_COMPRESS, 0, Q, B, q, as);
    }
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
  TLR_REQUIRE(!oz_timeout_flag(ctx), TLR_ERR_TIMEOUT, "split product: a bounded device wait ran out");
  for (void* c : chunks) dfree(ctx, c);
  M->state = 0;
}

// ======================================================================== factorization (factor.cu)
namespace tlr {
// Ensure Urow[i] of F has room for `extra` more columns (grow by copy).
void ensure_ucap(tlr_ctx* ctx, tlr_mat* F, int i, int64_t extra) {
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
}  // namespace tlr
namespace tlr {

// Solve plans.  For a factor and a number of right-hand sides the sequence of the two triangular
// solves is fixed: per block column k (Algorithm 7) Z_k = L_kk^-1 X_k, T = Vcol_k^T Z_k,
// X_i -= U_ik T_ik (i > k); then (LDL^T) Z = D^-1 Z; then, for k descending, S_ik = U_ik^T X_i,
// Z_k -= Vcol_k S, X_k = L_kk^-T Z_k.  A plan holds the buffers and the device job tables of that
// sequence (built once), runs it directly the first time, and on later solves with the same nrhs
// replays it as a CUDA graph captured once (~6 nb launches become one graph launch).
struct SolvePlan {
  int nrhs = 0;
  int64_t np = 0;
  double *X = nullptr, *Z = nullptr, *T = nullptr;
  SkJob* djobs = nullptr;
  SkItem* ditems = nullptr;
  struct Step { int kind, off, n; };  // kind 0 NN, 1 TN, 2 D^-1 scaling; items [off, off + n)
  std::vector<Step> steps;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches = 0;
  int runs = 0;
};

static void plan_destroy(tlr_ctx* ctx, SolvePlan* P) {
  if (!P) return;
  if (P->exec) {
    cudaStreamSynchronize(ctx->main);  // no replay of the graph still in flight
    cudaGraphExecDestroy(P->exec);
  }
  dfree(ctx, P->X);
  dfree(ctx, P->Z);
  dfree(ctx, P->T);
  dfree(ctx, P->djobs);
  dfree(ctx, P->ditems);
  delete P;
}

void mat_drop_plans(tlr_ctx* ctx, tlr_mat* M) {
  for (SolvePlan* P : M->plans) plan_destroy(ctx, P);
  M->plans.clear();
}

static SolvePlan* plan_build(tlr_ctx* ctx, const tlr_mat* F, int nrhs) {
  const int nb = F->nb, b = F->b;
  auto* P = new SolvePlan();
  P->nrhs = nrhs;
  P->np = (int64_t)nb * b;
  const int64_t np = P->np;
  int64_t rmax = 1;
  for (int k = 0; k < nb; ++k) rmax = std::max<int64_t>(rmax, F->vlen[k]);
  try {
    P->X = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)np * nrhs));
    P->Z = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)np * nrhs));
    P->T = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)rmax * nrhs));
    std::vector<SkJob> jobs;
    std::vector<SkItem> items;
    auto step = [&](int kind, const std::vector<SkJob>& js) {
      if (js.empty()) return;
      const int i0 = (int)items.size();
      sk_items(kind, js, (int)jobs.size(), items);
      P->steps.push_back({kind, i0, (int)items.size() - i0});
      jobs.insert(jobs.end(), js.begin(), js.end());
    };
    double *X = P->X, *Z = P->Z, *T = P->T;
    const int ld = (int)np;
    for (int k = 0; k < nb; ++k) {  // forward: L Z = X
      double* Zk = Z + (size_t)k * b;
      step(0, {SkJob{F->dinv + (size_t)k * b * b, X + (size_t)k * b, Zk, b, ld, ld, b, b, 1, 1.0, 0.0}});
      const int Rk = (int)F->vlen[k];
      if (Rk == 0) continue;
      step(1, {SkJob{F->Vcol[k], Zk, T, b, ld, Rk, Rk, b, 0, 1.0, 0.0}});
      std::vector<SkJob> upd;
      for (int i = k + 1; i < nb; ++i) {
        const int r = F->rank[ix(F, i, k)];
        if (r > 0) upd.push_back(SkJob{Uptr(F, i, k), T + F->voff[ix(F, i, k)], X + (size_t)i * b, b, Rk, ld, b, r, 0,
                                       -1.0, 1.0});
      }
      step(0, upd);
    }
    if (F->state == 2) P->steps.push_back({2, 0, 0});
    for (int k = nb - 1; k >= 0; --k) {  // backward: L^T X = Z
      double* Zk = Z + (size_t)k * b;
      const int Rk = (int)F->vlen[k];
      if (Rk > 0) {
        std::vector<SkJob> prj;
        for (int i = k + 1; i < nb; ++i) {
          const int r = F->rank[ix(F, i, k)];
          if (r > 0) prj.push_back(SkJob{Uptr(F, i, k), X + (size_t)i * b, T + F->voff[ix(F, i, k)], b, ld, Rk, r, b, 0,
                                         1.0, 0.0});
        }
        step(1, prj);
        step(0, {SkJob{F->Vcol[k], T, Zk, b, Rk, ld, b, Rk, 0, -1.0, 1.0}});
      }
      step(1, {SkJob{F->dinv + (size_t)k * b * b, Zk, X + (size_t)k * b, b, ld, ld, b, b, 1, 1.0, 0.0}});
    }
    P->djobs = static_cast<SkJob*>(dalloc(ctx, sizeof(SkJob) * std::max<size_t>(jobs.size(), 1)));
    P->ditems = static_cast<SkItem*>(dalloc(ctx, sizeof(SkItem) * std::max<size_t>(items.size(), 1)));
    // through the pinned upload ring (no host synchronization), then into the plan's own arrays
    auto put = [&](void* dst, const void* src, size_t bytes) {
      const size_t chunk = (size_t)16 << 20;
      for (size_t o = 0; o < bytes; o += chunk) {
        const size_t n = std::min(chunk, bytes - o);
        const void* d = upload(ctx, static_cast<const char*>(src) + o, n);
        TLR_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + o, d, n, cudaMemcpyDeviceToDevice, ctx->stream));
      }
    };
    put(P->djobs, jobs.data(), sizeof(SkJob) * jobs.size());
    put(P->ditems, items.data(), sizeof(SkItem) * items.size());
  } catch (...) {
    plan_destroy(ctx, P);
    throw;
  }
  return P;
}

static void plan_run(tlr_ctx* ctx, const tlr_mat* F, const SolvePlan* P) {
  for (const auto& s : P->steps) {
    if (s.kind == 2)
      scale_rows(ctx, (int)P->np, P->nrhs, F->dvec, 1, P->Z, (int)P->np, P->Z, (int)P->np);
    else
      sk_gemm(ctx, s.kind, P->djobs, P->ditems + s.off, s.n, P->nrhs);
  }
}

// Runs the plan on ctx->stream: directly the first time, as a captured graph afterwards.
static void plan_exec(tlr_ctx* ctx, const tlr_mat* F, SolvePlan* P) {
  if (P->runs++ == 0) {
    plan_run(ctx, F, P);
    return;
  }
  if (!P->exec) {
    if (!ctx->capture) TLR_CUDA(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    const int prof = ctx->prof;
    const int64_t l0 = ctx->launches;
    ctx->stream = ctx->capture;
    ctx->prof = 0;  // no profiling events inside the graph
    cudaGraph_t g = nullptr;
    TLR_CUDA(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
    try {
      plan_run(ctx, F, P);
    } catch (...) {
      cudaStreamEndCapture(ctx->capture, &g);
      if (g) cudaGraphDestroy(g);
      ctx->stream = saved;
      ctx->prof = prof;
      throw;
    }
    ctx->stream = saved;
    ctx->prof = prof;
    P->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    TLR_CUDA(cudaStreamEndCapture(ctx->capture, &g));
    const cudaError_t e = cudaGraphInstantiate(&P->exec, g, 0);
    cudaGraphDestroy(g);
    TLR_CUDA(e);
  }
  TLR_CUDA(cudaGraphLaunch(P->exec, ctx->stream));
  ctx->launches += P->graph_launches;
}

static SolvePlan* plan_for(tlr_ctx* ctx, tlr_mat* F, int nrhs) {
  for (size_t u = 0; u < F->plans.size(); ++u)
    if (F->plans[u]->nrhs == nrhs) {
      SolvePlan* P = F->plans[u];
      F->plans.erase(F->plans.begin() + u);
      F->plans.push_back(P);  // most recently used last
      return P;
    }
  constexpr size_t MAX_PLANS = 4;
  if (F->plans.size() >= MAX_PLANS) {
    plan_destroy(ctx, F->plans.front());
    F->plans.erase(F->plans.begin());
  }
  SolvePlan* P = plan_build(ctx, F, nrhs);
  F->plans.push_back(P);
  return P;
}

}  // namespace tlr

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

namespace tlr {
bool factor_opts_ok(const tlr_opts& o, int ldl, int64_t N, int b) {
  if (o.bs < 1 || o.bs > 64 || o.bs > b) return false;
  if (o.precision < TLR_PREC_FP64 || o.precision > TLR_PREC_MIXED) return false;
  if (o.compensation < TLR_COMP_NONE || o.compensation > TLR_COMP_MODCHOL) return false;
  if (o.compensation == TLR_COMP_MODCHOL && (ldl || b > 2048)) return false;  // Algorithm 8: Cholesky
  if (o.pivot < TLR_PIVOT_NONE || o.pivot > TLR_PIVOT_FROBENIUS) return false;
  if (o.pivot != TLR_PIVOT_NONE &&  // Algorithm 9: Cholesky, FP64, no padded tile to move
      (ldl || o.precision != TLR_PREC_FP64 || N % b != 0 ||
       (o.compensation != TLR_COMP_NONE && o.compensation != TLR_COMP_SHIFT)))
    return false;
  return true;
}
}  // namespace tlr

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

tlr_status tlr_create(tlr_ctx** out, int device, size_t hbm_budget, void* stream, tlr_alloc_fn alloc,
                      tlr_free_fn free_fn, void* user) {
  if (!out || ((alloc == nullptr) != (free_fn == nullptr))) return TLR_ERR_ARG;
  tlr_ctx* ctx = nullptr;
  ABI_BEGIN
  ctx = new tlr_ctx();
  ctx->device = device;
  ctx->hbm_budget = hbm_budget;
  TLR_CUDA(cudaSetDevice(device));
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->main = ctx->stream;
  {  // the side stream carries the diagonal tile's dependent chain (the column's trsm waits for it): its
     // CTAs are scheduled ahead of the main stream's when SMs free up
    int lo = 0, hi = 0;
    TLR_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    TLR_CUDA(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi));
  }
  TLR_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  TLR_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  ctx->alloc = alloc;
  ctx->free_fn = free_fn;
  ctx->user = user;
  TLR_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
  ctx->ring_cap = 64ull << 20;
  TLR_CUDA(cudaMallocHost(&ctx->pinned, ctx->ring_cap));
  ctx->djobs = static_cast<char*>(dalloc(ctx, ctx->ring_cap));
  if (const char* path = getenv("TLR_SITE_PROFILE")) ctx->site_out = fopen(path, "a");
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
  server_destroy(ctx);
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->side);
  if (ctx->site_out) {
    site_report(ctx);
    fclose(ctx->site_out);
    for (auto& v : ctx->sev)
      for (auto e : v) cudaEventDestroy(e);
  }
  dfree(ctx, ctx->djobs);
  dfree(ctx, ctx->scratch);
  dfree(ctx, ctx->scratch_side);
  dfree(ctx, ctx->split_ctr[0]);
  dfree(ctx, ctx->split_ctr[1]);
  dfree(ctx, ctx->orth_bar);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->hstatus) cudaFreeHost(ctx->hstatus);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
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
      kern->type != TLR_KERNEL_EXP || !(kern->nugget > -1.0))
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
      kern->type != TLR_KERNEL_EXP || !(kern->nugget > -1.0))
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
  M->plans.clear();  // plans belong to the source
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


static tlr_status check_factor_args(const tlr_mat* A, double eps, const tlr_opts& o, int ldl) {
  if (!A || !(eps > 0)) return TLR_ERR_ARG;
  if (A->state != 0) return TLR_ERR_STATE;
  return tlr::factor_opts_ok(o, ldl, A->N, A->b) ? TLR_OK : TLR_ERR_ARG;
}

static tlr_status factor_abi(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* opts, int ldl) {
  if (!ctx) return TLR_ERR_ARG;
  tlr_opts o = opts_or_default(opts);
  const tlr_status c = check_factor_args(A, eps, o, ldl);
  if (c != TLR_OK) return c;
  ABI_BEGIN
  std::vector<tlr_status> st;
  factor_batch(ctx, {A}, {eps}, {o}, ldl, st);
  return st[0];
  ABI_END
}

tlr_status tlr_factor_batch(tlr_ctx* ctx, int count, tlr_mat** A, const double* eps, const tlr_opts* opts, int ldl,
                            tlr_status* status) {
  if (!ctx || count < 0 || (count > 0 && (!A || !eps || !status))) return TLR_ERR_ARG;
  std::vector<tlr_mat*> mats;
  std::vector<double> ev;
  std::vector<tlr_opts> ov;
  std::vector<int> idx;
  for (int m = 0; m < count; ++m) {
    tlr_opts o = opts_or_default(opts ? &opts[m] : nullptr);
    status[m] = check_factor_args(A[m], eps[m], o, ldl);
    if (status[m] != TLR_OK) continue;
    mats.push_back(A[m]);
    ev.push_back(eps[m]);
    ov.push_back(o);
    idx.push_back(m);
  }
  if (mats.empty()) return TLR_OK;
  ABI_BEGIN
  std::vector<tlr_status> st;
  factor_batch(ctx, mats, ev, ov, ldl, st);
  for (size_t u = 0; u < idx.size(); ++u) status[idx[u]] = st[u];
  return TLR_OK;
  ABI_END
}

tlr_status tlr_potrf(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* o) { return factor_abi(ctx, A, eps, o, 0); }
tlr_status tlr_ldlt(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* o) { return factor_abi(ctx, A, eps, o, 1); }

tlr_status tlr_solve(tlr_ctx* ctx, const tlr_mat* F, int nrhs, double* B, int64_t ldb) {
  if (!ctx || !F || !B || nrhs < 0 || ldb < F->N) return TLR_ERR_ARG;
  if (F->state != 1 && F->state != 2) return TLR_ERR_STATE;
  if (nrhs == 0) return TLR_OK;
  ABI_BEGIN
  // right-hand sides in groups of at most 32 (one plan each)
  tlr_mat* Fm = const_cast<tlr_mat*>(F);  // the plan cache is not part of the factor's value
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int nc = std::min(32, nrhs - c0);
    double* Bc = B + (size_t)c0 * ldb;
    SolvePlan* P = plan_for(ctx, Fm, nc);
    permute_rows(ctx, F->N, nc, F->dperm, 1, Bc, ldb, P->X, P->np, P->np);
    plan_exec(ctx, F, P);
    permute_rows(ctx, F->N, nc, F->dperm, 0, P->X, P->np, Bc, ldb, P->np);
  }
  return TLR_OK;
  ABI_END
}

tlr_status tlr_pcg(tlr_ctx* ctx, const tlr_mat* A, const tlr_mat* F, int nrhs, const double* B, int64_t ldb,
                   double* X, int64_t ldx, double tol, int maxit, int* iters, double* relres) {
  if (!ctx || !A || !F || !B || !X || !iters || !relres || nrhs < 0 || !(tol > 0) || maxit < 0) return TLR_ERR_ARG;
  if (A->N != F->N || ldb < A->N || ldx < A->N || A->N > INT32_MAX) return TLR_ERR_ARG;
  if (A->state != 0 || (F->state != 1 && F->state != 2)) return TLR_ERR_STATE;
  if (nrhs == 0) return TLR_OK;
  ABI_BEGIN
  const int64_t n = A->N;
  auto check = [](tlr_status st, const char* what) {
    if (st != TLR_OK) throw Error(st, what);
  };
  Buf bR(ctx), bP(ctx), bQ(ctx), bZ(ctx), bS(ctx);
  double* R = bR.need<double>((size_t)n * nrhs);
  double* P = bP.need<double>((size_t)n * nrhs);
  double* Q = bQ.need<double>((size_t)n * nrhs);
  double* Z = bZ.need<double>((size_t)n * nrhs);
  double* sc = bS.need<double>((size_t)5 * nrhs);  // |b|^2, (r, z) twice, (p, A p), |r|^2 per column
  double* bn2 = sc;
  double* rz[2] = {sc + nrhs, sc + 2 * nrhs};
  double* pq = sc + 3 * nrhs;
  double* rr = sc + 4 * nrhs;
  const size_t cb = sizeof(double) * (size_t)n;
  TLR_CUDA(cudaMemset2DAsync(X, sizeof(double) * ldx, 0, cb, nrhs, ctx->stream));
  TLR_CUDA(cudaMemcpy2DAsync(R, cb, B, sizeof(double) * ldb, cb, nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  coldot(ctx, n, nrhs, B, ldb, B, ldb, bn2);
  double* h = static_cast<double*>(host_status(ctx, sizeof(double) * nrhs));
  d2h_sync(ctx, h, bn2, sizeof(double) * nrhs);
  std::vector<double> hb(h, h + nrhs);
  std::vector<int> act(nrhs);
  int nact = 0;
  for (int c = 0; c < nrhs; ++c) {
    act[c] = hb[c] > 0.0;  // a zero right-hand side has x = 0 after 0 iterations
    nact += act[c];
    iters[c] = 0;
  }
  // z0 = M^-1 r0, p0 = z0
  TLR_CUDA(cudaMemcpyAsync(Z, R, cb * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  if (nact > 0) check(tlr_solve(ctx, F, nrhs, Z, n), "pcg: preconditioner solve");
  TLR_CUDA(cudaMemcpyAsync(P, Z, cb * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  coldot(ctx, n, nrhs, R, n, Z, n, rz[0]);
  int cur = 0;
  for (int it = 1; it <= maxit && nact > 0; ++it) {
    check(tlr_matvec(ctx, A, TLR_OP_A, nrhs, P, n, Q, n), "pcg: operator product");
    coldot(ctx, n, nrhs, P, n, Q, n, pq);
    const int* da = static_cast<const int*>(upload(ctx, act.data(), sizeof(int) * nrhs));
    pcg_update_xr(ctx, n, nrhs, rz[cur], pq, da, X, ldx, P, R, Q, n);
    coldot(ctx, n, nrhs, R, n, R, n, rr);
    d2h_sync(ctx, h, rr, sizeof(double) * nrhs);
    for (int c = 0; c < nrhs; ++c)
      if (act[c] && (std::sqrt(h[c]) <= tol * std::sqrt(hb[c]) || it == maxit)) {
        act[c] = 0;
        iters[c] = it;
        --nact;
      }
    if (nact == 0) break;
    TLR_CUDA(cudaMemcpyAsync(Z, R, cb * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
    check(tlr_solve(ctx, F, nrhs, Z, n), "pcg: preconditioner solve");
    coldot(ctx, n, nrhs, R, n, Z, n, rz[1 - cur]);
    da = static_cast<const int*>(upload(ctx, act.data(), sizeof(int) * nrhs));
    pcg_update_p(ctx, n, nrhs, rz[1 - cur], rz[cur], da, Z, P, n);
    cur = 1 - cur;
  }
  // true residual |b - A x| / |b|
  check(tlr_matvec(ctx, A, TLR_OP_A, nrhs, X, ldx, Q, n), "pcg: operator product");
  TLR_CUDA(cudaMemcpy2DAsync(R, cb, B, sizeof(double) * ldb, cb, nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  axpy_matrix(ctx, (int)n, nrhs, -1.0, Q, (int)n, R, (int)n);
  coldot(ctx, n, nrhs, R, n, R, n, rr);
  d2h_sync(ctx, h, rr, sizeof(double) * nrhs);
  for (int c = 0; c < nrhs; ++c) relres[c] = hb[c] > 0.0 ? std::sqrt(h[c] / hb[c]) : 0.0;
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
  if (!ctx || !kernel_product_args_ok(pts, kern, X, Y, N, d, nrhs, ldx, ldy)) return TLR_ERR_ARG;
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
  std::vector<int> q;
  AraStats as;
  ara_dense_run(ctx, nops, n, T, bs, eps, seed, stream, k, Q, Bout, q, as);
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
  std::vector<DenseTile> t{DenseTile{A, nullptr, di, nullptr, n, lda}};
  dense_factor_batch(ctx, t, 0, tmp);
  d2h_sync(ctx, info, di, sizeof(int));
  return TLR_OK;
  ABI_END
}

tlr_status tlr_dense_modchol(tlr_ctx* ctx, int n, double* A, int lda, int* modified, int* info) {
  if (!ctx || !A || n < 0 || n > 2048 || lda < n || !info || !modified) return TLR_ERR_ARG;
  ABI_BEGIN
  Buf bi(ctx), tmp(ctx), cp(ctx), work(ctx);
  int* di = bi.need<int>(1);
  double* A0 = cp.need<double>(std::max<size_t>((size_t)n * n, 1));
  copy_matrix(ctx, n, n, A, lda, A0, n);
  TLR_CUDA(cudaMemsetAsync(di, 0xff, sizeof(int), ctx->stream));
  std::vector<DenseTile> t{DenseTile{A, nullptr, di, nullptr, n, lda}};
  dense_factor_batch(ctx, t, 0, tmp);
  d2h_sync(ctx, info, di, sizeof(int));
  *modified = 0;
  if (*info >= 0) {  // not positive definite: Algorithm 8 on the input
    *modified = 1;
    copy_matrix(ctx, n, n, A0, n, A, lda);
    modified_cholesky_tile(ctx, n, A, lda, nullptr, di, work, tmp);
    d2h_sync(ctx, info, di, sizeof(int));
  }
  return TLR_OK;
  ABI_END
}

tlr_status tlr_trim_tiles(tlr_ctx* ctx, int ntiles, int b, int r, const double* Q, const double* B, double eps,
                          double* Qout, double* Bout, int* rank) {
  if (!ctx || ntiles < 0 || b < 1 || r < 0 || r > b || !(eps > 0) || (ntiles > 0 && !rank) ||
      (ntiles > 0 && r > 0 && (!Q || !B || !Qout || !Bout)))
    return TLR_ERR_ARG;
  if (!trim_fits(b)) return TLR_ERR_LIMIT;
  ABI_BEGIN
  std::vector<int> rk(ntiles, 0);
  if (r > 0 && ntiles > 0) {
    std::vector<TrimTile> tl(ntiles);
    for (int t = 0; t < ntiles; ++t) tl[t] = TrimTile{B + (size_t)t * b * r, r};
    Buf work(ctx);
    std::vector<double*> Zs;
    trim_tiles(ctx, b, tl, eps, rk, Zs, work);
    const size_t bytes = sizeof(double) * (size_t)ntiles * b * r;
    TLR_CUDA(cudaMemsetAsync(Qout, 0, bytes, ctx->stream));
    TLR_CUDA(cudaMemsetAsync(Bout, 0, bytes, ctx->stream));
    std::vector<GemmJob<double>> jobs;
    for (int t = 0; t < ntiles; ++t) {
      if (rk[t] == 0) continue;
      const size_t o = (size_t)t * b * r;
      jobs.push_back(job<double>(NN, b, rk[t], Q + o, b, Zs[t], r, r, Qout + o, b, 1.0, 0.0));
      jobs.push_back(job<double>(NN, b, rk[t], B + o, b, Zs[t], r, r, Bout + o, b, 1.0, 0.0));
    }
    gemm<double>(ctx, NN, jobs);
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  for (int t = 0; t < ntiles; ++t) rank[t] = rk[t];
  return TLR_OK;
  ABI_END
}

tlr_status tlr_trim(tlr_ctx* ctx, tlr_mat* A, double eps) {
  if (!ctx || !A || !(eps > 0)) return TLR_ERR_ARG;
  if (A->state != 0 && A->state != 1 && A->state != 2) return TLR_ERR_STATE;
  if (!trim_fits(A->b)) return TLR_ERR_LIMIT;
  ABI_BEGIN
  trim_matrix(ctx, A, eps);
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
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
  std::vector<DenseTile> t{DenseTile{A, d, di, nullptr, n, lda}};
  dense_factor_batch(ctx, t, 1, tmp);
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

tlr_status tlr_split_product(tlr_ctx* ctx, int trans, int n, int ncols, const double* T, const double* X, int ldx,
                             double* C, int ldc) {
  if (!ctx || !T || !X || !C || n <= 0 || ncols < 0 || ldx < n || ldc < n || trans < 0 || trans > 2) return TLR_ERR_ARG;
  if (n % 16 != 0) return TLR_ERR_LIMIT;
  if (ncols == 0) return TLR_OK;
  ABI_BEGIN
  Buf bm(ctx), bS(ctx), be(ctx), bx(ctx), bex(ctx);
  unsigned long long* tmax = bm.need<unsigned long long>(1);
  oz_absmax(ctx, 1, (int64_t)n * n, T, tmax);
  int8_t* Sc = bS.need<int8_t>((size_t)16 * n * n);
  int8_t* Sr = Sc + (size_t)8 * n * n;
  int* eT = be.need<int>(1);
  oz_split_tiles(ctx, 1, n, T, tmax, Sc, Sr, eT);
  int8_t* Xs = bx.need<int8_t>((size_t)8 * n * ncols);
  int* ex = bex.need<int>((size_t)ncols);
  std::vector<OzColJob> cj{OzColJob{X, Xs, ex, ldx, ncols, 0, n}};
  oz_split_cols(ctx, cj);
  std::vector<OzJob> jobs{OzJob{trans == 1 ? Sc : Sr, Xs, eT, ex, C, (size_t)n * n, (size_t)n * ncols, n, ldc, n, ncols, n}};
  if (trans == 2) {  // T X with T read by columns: A(m, k) = Sc[m + k n]
    jobs[0].A = Sc;
    jobs[0].acol = 1;
  }
  oz_gemm(ctx, jobs);
  if (oz_timeout_flag(ctx)) return TLR_ERR_TIMEOUT;
  return TLR_OK;
  ABI_END
}

tlr_status tlr_split_planes(tlr_ctx* ctx, int64_t* counts, double* bytes, int reset) {
  if (!ctx) return TLR_ERR_ARG;
  ABI_BEGIN
  unsigned long long st[10];
  oz_stats(ctx, st, reset);
  if (counts)
    for (int s = 0; s < 9; ++s) counts[s] = s == 0 ? 0 : (int64_t)st[s];
  if (bytes) *bytes = (double)st[9];
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

tlr_status tlr_gemm_stats(tlr_ctx* ctx, int enable, double* ms, double* flops, double* bytes, int64_t* launches) {
  if (!ctx) return TLR_ERR_ARG;
  ABI_BEGIN
  kprof_flush(ctx);
  for (int f = 0; f < TLR_GEMM_FAMILIES; ++f) {
    if (ms) ms[f] = ctx->kfam_ms[f];
    if (flops) flops[f] = ctx->kfam_flops[f];
    if (bytes) bytes[f] = ctx->kfam_bytes[f];
    if (launches) launches[f] = ctx->kfam_launches[f];
    ctx->kfam_ms[f] = 0; ctx->kfam_flops[f] = 0; ctx->kfam_bytes[f] = 0; ctx->kfam_launches[f] = 0;
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
