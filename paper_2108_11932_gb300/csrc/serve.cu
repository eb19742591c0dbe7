// Serving queue of the library: tlr_submit / tlr_progress / tlr_poll.
//
// A request is one covariance matrix (points, kernel, tile size, threshold) to build, factor
// (Algorithm 6 or 10), solve with its right-hand sides (Algorithm 7 and its transpose) and take
// the log determinant of.  Admission compares the context's device bytes in use (every library
// allocation is counted) plus the next request's estimated footprint with the context's budget;
// admitted requests join one tlr_session, so their column steps share launches with the
// factorizations already in flight, and a request gets the same result alone or in the mix.
// A factorization that loses definiteness is rebuilt and refactored once with the diagonal
// shift eps I of Section 5.1.  Everything here is scheduling: the GPU work is the library's.
#include <math.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <map>

#include "internal.h"

namespace tlr {

namespace {
using Clock = std::chrono::steady_clock;
double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }
}  // namespace

struct Server {
  struct Req {
    tlr_request rq{};
    std::vector<double> pts, rhs, x;
    tlr_mat* A = nullptr;
    int sticket = -1;
    int state = 0;  // 0 queued, 1 in flight, 2 done
    tlr_result res{};
    Clock::time_point t_submit, t_admit;
  };
  tlr_ctx* ctx;
  tlr_session* S = nullptr;
  int bs = -1;
  uint64_t next = 1;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Req> reqs;
  int in_flight = 0;
  explicit Server(tlr_ctx* c) : ctx(c) {}
  ~Server() {
    for (auto& kv : reqs)
      if (kv.second.A) tlr_free(ctx, kv.second.A);
    if (S) tlr_session_destroy(S);
  }

  // Device bytes of a request while it is resident: the dense diagonal tiles of A and of its factor
  // and the inverses of the factor's diagonal tiles (3 N b), the low-rank factors of A and of L at a
  // mean rank estimated from eps and the dimension (exponential kernels: ranks grow like log(1/eps),
  // roughly twice as fast in 3D), their 7-bit chunk planes for the tensor-core products, the ARA
  // workspace, the points and right-hand sides.
  static size_t footprint(const tlr_request& r) {
    const double nb = std::ceil((double)r.N / r.b);
    const double rbar = std::max(4.0, 3.0 * std::log10(1.0 / r.eps)) * (r.d >= 3 ? 2.0 : 1.0);
    const double lowrank = 2.0 * 2.0 * (nb * (nb - 1.0) / 2.0) * r.b * rbar;  // A and L, U and V
    const double planes = 3.0 * (nb * (nb - 1.0) / 2.0) * r.b * rbar;         // int8: 3 bytes per 8
    const double work = nb * r.b * (double)(r.b + 64);
    return (size_t)(8.0 * (3.0 * nb * r.b * r.b + lowrank + work + (double)r.N * (r.d + r.nrhs)) + planes);
  }

  tlr_status build(Req& q, bool shifted) {
    tlr_opts o = q.rq.opts;
    if (shifted) {
      o.compensation = TLR_COMP_SHIFT;
      o.shift = q.rq.eps;
    }
    tlr_status st = tlr_compress(ctx, q.pts.data(), q.rq.N, q.rq.d, &q.rq.kernel, q.rq.b, q.rq.eps, &o, &q.A);
    if (st != TLR_OK) return st;
    return tlr_session_add(S, q.A, q.rq.eps, &o, q.rq.ldl, &q.sticket);
  }

  void finish(Req& q, tlr_status st) {
    q.state = 2;
    q.res.done = 1;
    q.res.status = st;
    q.res.run_s = secs(q.t_admit, Clock::now());
    if (q.A) tlr_free(ctx, q.A);
    q.A = nullptr;
    --in_flight;
  }

  void complete(Req& q) {  // solve, logdet, release
    tlr_info inf{};
    tlr_get_info(q.A, &inf);
    q.res.bytes = inf.bytes;
    q.res.mean_rank = inf.mean_rank;
    tlr_status st = TLR_OK;
    if (q.rq.nrhs > 0) {
      const size_t n = (size_t)q.rq.N * q.rq.nrhs;
      double* B = static_cast<double*>(dalloc(ctx, sizeof(double) * n));
      TLR_CUDA(cudaMemcpyAsync(B, q.rhs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
      st = tlr_solve(ctx, q.A, q.rq.nrhs, B, q.rq.N);
      if (st == TLR_OK) {
        q.x.resize(n);
        TLR_CUDA(cudaMemcpyAsync(q.x.data(), B, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
        TLR_CUDA(cudaStreamSynchronize(ctx->stream));
      }
      dfree(ctx, B);
      q.rhs.clear();
      q.rhs.shrink_to_fit();
    }
    if (st == TLR_OK) st = tlr_logdet(ctx, q.A, &q.res.logdet, &q.res.sign);
    finish(q, st);
  }

  void progress() {
    if (!S) TLR_REQUIRE(tlr_session_create(ctx, &S) == TLR_OK, TLR_ERR_CUDA, "serving: session");
    // 1. admission in submission order
    while (!queue.empty()) {
      Req& q = reqs.at(queue.front());
      if (in_flight > 0 && ctx->hbm_budget > 0 && ctx->live_bytes + footprint(q.rq) > ctx->hbm_budget) break;
      queue.pop_front();
      q.state = 1;
      q.t_admit = Clock::now();
      q.res.wait_s = secs(q.t_submit, q.t_admit);
      ++in_flight;
      const tlr_status st = build(q, false);
      if (st != TLR_OK) finish(q, st);
    }
    if (in_flight == 0) return;
    // 2. one column step of everything in flight
    int unfinished = 0;
    const tlr_status st = tlr_session_step(S, &unfinished);
    TLR_REQUIRE(st == TLR_OK, st, "serving: column step failed");
    // 3. finished factorizations
    for (auto& kv : reqs) {
      Req& q = kv.second;
      if (q.state != 1 || q.sticket < 0) continue;
      int fin = 0;
      tlr_status fst = TLR_OK;
      tlr_session_poll(S, q.sticket, &fin, &fst);
      if (!fin) continue;
      q.sticket = -1;
      if (fst == TLR_ERR_NOT_SPD && !q.res.retried && q.rq.opts.compensation == TLR_COMP_NONE) {
        tlr_free(ctx, q.A);
        q.A = nullptr;
        q.res.retried = 1;
        const tlr_status bst = build(q, true);
        if (bst != TLR_OK) finish(q, bst);
        continue;
      }
      if (fst != TLR_OK) finish(q, fst);
      else complete(q);
    }
  }
};

void server_destroy(tlr_ctx* ctx) {
  delete ctx->server;
  ctx->server = nullptr;
}

}  // namespace tlr

using namespace tlr;

extern "C" {

tlr_status tlr_submit(tlr_ctx* ctx, const tlr_request* r, uint64_t* ticket) {
  if (!ctx || !r || !ticket || !r->points || r->N <= 0 || r->d < 1 || r->d > 3 || r->b < 1 || !(r->eps > 0) ||
      r->nrhs < 0 || r->nrhs > 1024 || (r->nrhs > 0 && !r->rhs) || r->ldl < 0 || r->ldl > 1 ||
      r->kernel.type != TLR_KERNEL_EXP || !(r->kernel.ell > 0) || !(r->kernel.nugget > -1.0))
    return TLR_ERR_ARG;
  tlr_opts ro = r->opts;
  if (ro.bs <= 0) ro.bs = 16;
  const int bs = ro.bs;
  if (!tlr::factor_opts_ok(ro, r->ldl, r->N, r->b)) return TLR_ERR_ARG;
  try {
    if (!ctx->server) ctx->server = new Server(ctx);
    Server& sv = *ctx->server;
    if (sv.bs >= 0 && bs != sv.bs) return TLR_ERR_ARG;  // one ARA block width per queue
    sv.bs = bs;
    const uint64_t t = sv.next++;
    Server::Req& q = sv.reqs[t];
    q.rq = *r;
    q.rq.opts.bs = bs;
    q.pts.assign(r->points, r->points + (size_t)r->N * r->d);
    if (r->nrhs > 0) q.rhs.assign(r->rhs, r->rhs + (size_t)r->N * r->nrhs);
    q.rq.points = nullptr;
    q.rq.rhs = nullptr;
    q.t_submit = Clock::now();
    sv.queue.push_back(t);
    *ticket = t;
    return TLR_OK;
  } catch (const std::bad_alloc&) {
    return TLR_ERR_NOMEM;
  } catch (...) {
    return TLR_ERR_CUDA;
  }
}

tlr_status tlr_progress(tlr_ctx* ctx, int* queued, int* in_flight) {
  if (!ctx) return TLR_ERR_ARG;
  try {
    if (ctx->server) ctx->server->progress();
    if (queued) *queued = ctx->server ? (int)ctx->server->queue.size() : 0;
    if (in_flight) *in_flight = ctx->server ? ctx->server->in_flight : 0;
    return TLR_OK;
  } catch (const tlr::Error& e) {
    fprintf(stderr, "[tlr] %s\n", e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    return TLR_ERR_NOMEM;
  } catch (...) {
    return TLR_ERR_CUDA;
  }
}

tlr_status tlr_poll(tlr_ctx* ctx, uint64_t ticket, tlr_result* res, double* x, int64_t ldx) {
  if (!ctx || !res || !ctx->server) return TLR_ERR_ARG;
  Server& sv = *ctx->server;
  auto it = sv.reqs.find(ticket);
  if (it == sv.reqs.end()) return TLR_ERR_ARG;
  Server::Req& q = it->second;
  if (q.state != 2) {
    memset(res, 0, sizeof(*res));
    return TLR_OK;
  }
  if (x && ldx < q.rq.N) return TLR_ERR_ARG;
  *res = q.res;
  if (x && q.res.status == TLR_OK)
    for (int c = 0; c < q.rq.nrhs; ++c)
      memcpy(x + (size_t)c * ldx, q.x.data() + (size_t)c * q.rq.N, sizeof(double) * q.rq.N);
  sv.reqs.erase(it);
  return TLR_OK;
}

}  // extern "C"
