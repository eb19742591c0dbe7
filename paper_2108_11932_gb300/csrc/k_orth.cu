// Fused orthogonalization round of the batched ARA.
//
// Algorithm 1 orthogonalizes each new sample block Y (n x bs) against the basis Q (n x q) found so far
// and then within itself; Algorithm 5 runs this for every operand of the dynamic batch.  Here one round
// of every slot is one launch:
//   first pass (pass = 0):   Y <- Y - Q (Q^T Y);  G = Y^T Y;  M1 = CholQR(G) with the convergence test;
//                            W = Y M1
//   second pass (pass = 1):  W <- W - Q (Q^T W);  G = W^T W;  M2 = CholQR(G) on the kept columns;
//                            Q[:, q:q+bs] = W M2
// (block classical Gram-Schmidt with re-orthogonalization, BCGS2, and Cholesky-QR with dropping, the
// same steps and decisions as the chain of batched products and k_cholqr_reg launches it replaces).
//
// The FP64 unit bounds these products (2 DFMA per clock and SM), and a round in a column's tail has one
// to three slots, so every product is cut into units small enough to spread one slot over all SMs:
//   Q^T X    units of 8 basis columns x 64 rows (a row chunk); the partial sums of the chunks are added
//            in chunk order by the CTA that completes the column block (arrival ticket)
//   X - Q S  units of rb rows (8 to 64, from the slot's own q), each with its Gram partial X^T X; the CTA
//            that completes a 64-row chunk adds its units' partials in order, and the CTA that completes
//            the slot adds the chunks' in order and runs the Cholesky-QR
//   X M      row-local, any split
// Each CTA takes a contiguous range of a phase's units (over all slots), so one slot's units run on
// many SMs and a CTA rarely changes slot.  Phases are separated by grid-wide barriers (the grid is sized
// so that every CTA is resident).  Every sum runs in an order fixed by the slot's own shape (n, q),
// never by the launch it shares or by which CTA takes a unit, so a slot's result does not depend on the
// other slots of the round.  Every wait is bounded: a barrier that runs out sets g_orth_timeout, and the
// CTAs leave the kernel.
#include <math.h>

#include <cstring>

#include "cholqr.cuh"
#include "internal.h"

namespace tlr {

__device__ int g_orth_timeout = 0;

namespace {

constexpr int OR_T = 256;          // threads per CTA
constexpr int OR_CB = 8;           // basis columns per Q^T X unit
constexpr int OR_RC = 64;          // rows of a chunk (Q^T X units, Gram chunk partials, X M steps)
constexpr int OR_LD = OR_RC + 1;   // padded leading dimension of staged row blocks (odd: no bank conflicts)
constexpr unsigned long long OR_WAIT_NS = 2000000000ull;  // 2 s per barrier

struct OrthDev {     // one slot of the round
  const double* Q;   // n x q basis, ld n
  double* Qn;        // Q + q n: the round's new columns
  double* Y;         // n x bs sample block, projected in place
  double* W;         // n x bs
  double* Sp;        // partial Q^T X per row chunk: nrc blocks of q x bs (ld q)
  double* Sf;        // Q^T X, q x bs (ld q)
  double* Gp;        // Gram partials per rb-row unit: nrb x bs x bs
  double* Gc;        // Gram partials per 64-row chunk: nrc x bs x bs
  double* M;         // bs x bs factor of the current pass
  int* cnt;          // arrival tickets: ncb (column blocks), nrc (row chunks), 1 (slot); zero between launches
  int* st;           // {converged, kept}
  double* en;        // convergence norm
  double thr;
  int n, q, nrc, ncb, rb, nrb;
};
struct OrthHdr {
  int ns, pad;
  int total[4];      // units of the phases: Q^T X, X - Q S, X M of the first pass (slots with a basis), X M
  double tau;
};
static_assert(sizeof(OrthHdr) % 8 == 0 && sizeof(OrthDev) % 8 == 0, "table alignment");

// staged basis rows (doubles) and basis columns of S per step of X - Q S
constexpr int OR_QCAP = 4096;
template <int BS>
__host__ __device__ constexpr int or_scap() { return BS == 16 ? 256 : 128; }
// shared doubles of the largest phase (X - Q S with its Gram partials and Cholesky-QR)
template <int BS>
__host__ __device__ constexpr int or_smem() {
  return BS * OR_LD + 2 * OR_QCAP + or_scap<BS>() * (BS + 1) + BS * BS + BS * BS;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long gclock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier: bar[0] counts arrivals, bar[1] is the generation.  Returns false when the wait ran
// out or another CTA gave up (then the caller leaves the kernel).
__device__ bool grid_sync(unsigned* bar) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    const unsigned gen = ld_acquire(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = gclock();
      for (unsigned it = 0; ld_acquire(bar + 1) == gen; ++it) {
        if ((it & 31u) == 31u &&
            (*(volatile int*)&g_orth_timeout || gclock() - t0 > OR_WAIT_NS || it > (1u << 26))) {
          atomicExch(&g_orth_timeout, 1);
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// This CTA's contiguous range [u0, u1) of a phase's units, and the slot of u0 (the largest s with
// p[s] <= u0; slots without units have p[s] == p[s + 1]).
struct Range {
  int u0, u1, s;
};
__device__ __forceinline__ Range unit_range(const int* p, int ns, int total) {
  const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  Range R;
  R.u0 = min(total, (int)blockIdx.x * per);
  R.u1 = min(total, R.u0 + per);
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p[mid] <= R.u0) lo = mid;
    else hi = mid - 1;
  }
  R.s = lo;
  return R;
}
// slot of unit u >= the previous unit's, from the previous slot s
__device__ __forceinline__ int next_slot(const int* p, int ns, int s, int u) {
  while (s + 1 < ns && p[s + 1] <= u) ++s;
  return s;
}

// the Cholesky-QR as a call of its own: inlined into this kernel its register arrays went to local memory
template <int BS>
__device__ __noinline__ void cholqr_slot(const double* G, double* M, int* st, double* en, double thr, double tau,
                                         int first_pass, int nk_in) {
  cholqr_warp<BS>(G, M, st, en, thr, tau, first_pass, nk_in);
}

__device__ __forceinline__ bool converged(const OrthDev& D) { return __ldcg(D.st) != 0; }

// row r, column j of X M for rows staged column-major in Xs (ld ldx) and M (BS x BS) in Ms
template <int BS>
__device__ __forceinline__ double xm_entry(const double* Xs, int ldx, int r, const double* Ms, int j) {
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < BS; ++k) acc = fma(Xs[k * ldx + r], Ms[k + j * BS], acc);
  return acc;
}

// Arrival ticket: true in the CTA whose `add` arrivals bring the count to `target` (that CTA resets
// it).  The CTA barrier orders its threads' writes before thread 0's device-scope fence and atomic (the
// fence is cumulative), and thread 0's fence after a completing count orders the partials written by
// the other CTAs before this CTA's reads of them.
__device__ __forceinline__ bool ticket(int* cnt, int add, int target) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(cnt, add) + add == target;
    if (last) {
      *cnt = 0;
      __threadfence();
    }
  }
  __syncthreads();
  return last != 0;
}

// S = Q^T X (X = Y in pass 0, W in pass 1) for the slots with a basis.  Units (row chunk rc, column
// block cb), rc-major; a CTA takes up to QG consecutive units of one slot and chunk in one step (the rows
// of X staged once), and loads the next step's basis tile into registers while it computes.  Each output
// of a unit is the sum of two chains, rows 0-31 and 32-63 of the chunk, whatever the step holds.
template <int BS>
__device__ void phase_qtx(const OrthHdr& H, const OrthDev* J, const int* pa, int pass, double* sm) {
  constexpr int QG = 64 / BS;            // units per step
  constexpr int NQ = QG * OR_CB;         // basis columns per step
  constexpr int PT = NQ * BS / OR_T;     // outputs per thread
  constexpr int QPF = NQ * OR_RC / OR_T; // basis entries per thread of a step's tile
  static_assert(NQ * BS % OR_T == 0 && NQ * OR_RC % OR_T == 0, "step shape");
  double* Qs = sm;                 // NQ x OR_LD
  double* Xs = Qs + NQ * OR_LD;    // BS x OR_LD
  __shared__ int fin[QG];
  const int t = threadIdx.x;
  const Range R = unit_range(pa, H.ns, H.total[0]);
  if (R.u0 >= R.u1) return;
  struct Step {
    int s, rc, cb0, k;
    bool skip;
  };
  auto step_at = [&](int u, int s_from) {
    Step st;
    st.s = next_slot(pa, H.ns, s_from, u);
    const OrthDev& D = J[st.s];
    const int li = u - pa[st.s];
    st.rc = li / D.ncb;
    st.cb0 = li % D.ncb;
    st.k = min(min(R.u1 - u, QG), D.ncb - st.cb0);
    st.skip = pass && converged(D);
    return st;
  };
  double pf[QPF];
  auto load_tile = [&](const Step& st) {
    const OrthDev& D = J[st.s];
    const int c0 = st.cb0 * OR_CB, r0 = st.rc * OR_RC;
    const int nc = min(st.k * OR_CB, D.q - c0), nr = min(OR_RC, D.n - r0);
#pragma unroll
    for (int v = 0; v < QPF; ++v) {
      const int e = t + v * OR_T, r = e % OR_RC, cc = e / OR_RC;
      pf[v] = (r < nr && cc < nc) ? D.Q[(size_t)(r0 + r) + (size_t)(c0 + cc) * D.n] : 0.0;
    }
  };
  int u = R.u0, xs_slot = -1, xs_rc = -1;
  Step cur = step_at(u, R.s);
  if (!cur.skip) load_tile(cur);
  while (true) {
    const int un = u + cur.k;
    const bool more = un < R.u1;
    Step nxt = cur;
    if (more) nxt = step_at(un, cur.s);
    if (cur.skip) {
      if (more && !nxt.skip) load_tile(nxt);
    } else {
      const OrthDev& D = J[cur.s];
      const int rc = cur.rc, k = cur.k, c0 = cur.cb0 * OR_CB, r0 = rc * OR_RC, q = D.q;
      const int nc = min(k * OR_CB, q - c0), nr = min(OR_RC, D.n - r0);
      __syncthreads();  // the previous step's readers of the staged blocks are done
#pragma unroll
      for (int v = 0; v < QPF; ++v) {
        const int e = t + v * OR_T;
        Qs[(e / OR_RC) * OR_LD + e % OR_RC] = pf[v];
      }
      if (cur.s != xs_slot || rc != xs_rc) {
        const double* X = pass ? D.W : D.Y;
        for (int e = t; e < BS * OR_RC; e += OR_T) {
          const int r = e % OR_RC, jj = e / OR_RC;
          Xs[jj * OR_LD + r] = r < nr ? __ldcg(X + (size_t)(r0 + r) + (size_t)jj * D.n) : 0.0;
        }
        xs_slot = cur.s;
        xs_rc = rc;
      }
      if (more && !nxt.skip) load_tile(nxt);  // in flight during this step's products
      __syncthreads();
#pragma unroll
      for (int v = 0; v < PT; ++v) {
        const int o = t + v * OR_T, c = o / BS, j = o % BS;
        if (c < nc) {
          double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
          for (int r = 0; r < OR_RC / 2; ++r) {
            a0 = fma(Qs[c * OR_LD + r], Xs[j * OR_LD + r], a0);
            a1 = fma(Qs[c * OR_LD + r + OR_RC / 2], Xs[j * OR_LD + r + OR_RC / 2], a1);
          }
          D.Sp[(size_t)rc * q * BS + (c0 + c) + (size_t)j * q] = a0 + a1;
        }
      }
      __syncthreads();
      if (t < k) {  // arrival tickets of the step's column blocks (see ticket())
        const int cb = cur.cb0 + t;
        __threadfence();
        const bool l = atomicAdd(D.cnt + cb, 1) + 1 == D.nrc;
        if (l) {
          D.cnt[cb] = 0;
          __threadfence();
        }
        fin[t] = l;
      }
      __syncthreads();
      bool any = false;
      for (int i = 0; i < k; ++i) any |= fin[i] != 0;
      if (any) {
#pragma unroll
        for (int v = 0; v < PT; ++v) {  // completed column blocks: the sums in row-chunk order
          const int o = t + v * OR_T, c = o / BS, j = o % BS;
          if (c < nc && fin[c / OR_CB]) {
            double w = 0.0;
            for (int kk = 0; kk < D.nrc; ++kk) w += __ldcg(D.Sp + (size_t)kk * q * BS + (c0 + c) + (size_t)j * q);
            D.Sf[(c0 + c) + (size_t)j * q] = w;
          }
        }
      }
    }
    if (!more) break;
    u = un;
    cur = nxt;
  }
}

// 8-byte asynchronous copy global -> shared (zero-filled when !valid); the basis it is used for is not
// written by the kernel, so the L1-allocating form is safe
__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// X <- X - Q S on rb-row units and their Gram partials; the CTA completing a chunk adds the chunk's
// partials, the CTA completing the slot adds the chunks' and runs the Cholesky-QR.  A CTA takes up to a
// chunk of consecutive units of one slot in one step; the next step's first basis chunk is copied
// asynchronously into the other of two buffers while the step computes, and S stays staged across the
// steps of a slot when it fits one chunk.  In the second pass a slot without a basis forms its rows of
// W = Y M1 here (the first pass's X M phase skips it: no Q^T W needs the whole of W).
template <int BS>
__device__ void phase_project(const OrthHdr& H, const OrthDev* J, const int* pb, int pass, double* sm) {
  constexpr int SLD = BS + 1;                 // padded leading dimension of staged rows of S
  constexpr int MAXO = OR_RC * BS / OR_T;     // outputs per thread for a full chunk
  constexpr int GE = (BS * BS + OR_T - 1) / OR_T;  // Gram entries per thread per unit
  double* Xn = sm;                   // BS x OR_LD: the step's rows, column-major
  double* Qb[2] = {Xn + BS * OR_LD, Xn + BS * OR_LD + OR_QCAP};  // kc x rows (Y rows, ld OR_LD, without a basis)
  double* Ss = Qb[1] + OR_QCAP;      // kc x SLD
  double* Ms = Ss + or_scap<BS>() * SLD;  // BS x BS
  double* Gs = Ms + BS * BS;         // BS x BS
  static_assert(BS * OR_LD <= OR_QCAP, "Y rows fit the staging area");
  const int t = threadIdx.x;
  const Range R = unit_range(pb, H.ns, H.total[1]);
  if (R.u0 >= R.u1) return;
  struct Step {
    int s, blk0, k;
    bool skip;
  };
  auto step_at = [&](int u, int s_from) {
    Step st;
    st.s = next_slot(pb, H.ns, s_from, u);
    const OrthDev& D = J[st.s];
    const int bpc = OR_RC / D.rb;
    st.blk0 = u - pb[st.s];
    // units blk0 .. blk0 + k - 1 of one chunk, within the CTA's range
    st.k = min(min(R.u1 - u, bpc - st.blk0 % bpc), D.nrb - st.blk0);
    st.skip = pass && converged(D);
    return st;
  };
  auto kc_of = [](int q, int nr) { return max(2, min(min(or_scap<BS>(), OR_QCAP / nr), (q + 1) & ~1) & ~1); };
  // the first basis chunk of a step (Qs[cc * nr + r], zero past q) into buffer dst
  auto copy_chunk0 = [&](const Step& st, double* dst) {
    const OrthDev& D = J[st.s];
    const int q = D.q, r0 = st.blk0 * D.rb, nr = min(st.k * D.rb, D.n - r0);
    const int kq = min(kc_of(q, nr), q), ke = (kq + 1) & ~1;
    for (int e = t; e < ke * nr; e += OR_T) {
      const int r = e % nr, cc = e / nr;
      const bool ok = cc < kq;
      cp_async8(dst + e, D.Q + (ok ? (size_t)(r0 + r) + (size_t)cc * D.n : 0), ok);
    }
  };
  int u = R.u0, ss_slot = -1, qbuf = 0;  // ss_slot: the slot whose whole S is staged in Ss
  bool ready = false;                    // the current step's first chunk is in flight to Qb[qbuf]
  Step cur = step_at(u, R.s);
  while (true) {
    const int un = u + cur.k;
    const bool more = un < R.u1;
    Step nxt = cur;
    if (more) nxt = step_at(un, cur.s);
    if (!cur.skip) {
      const OrthDev& D = J[cur.s];
      const int RB = D.rb, bpc = OR_RC / RB, q = D.q, blk0 = cur.blk0, k = cur.k, rc = blk0 / bpc;
      const int r0 = blk0 * RB, nr = min(k * RB, D.n - r0);  // rows of the step
      double* X = pass ? D.W : D.Y;
      double* Qs = Qb[qbuf];
      const int kc = q > 0 ? kc_of(q, nr) : 2;
      const int kq0 = min(kc, q), ke0 = (kq0 + 1) & ~1;
      __syncthreads();  // the previous steps' readers of both buffers are done
      if (pass && q == 0) {
        for (int e = t; e < BS * BS; e += OR_T) Ms[e] = __ldcg(D.M + e);
        for (int e = t; e < BS * OR_RC; e += OR_T) {
          const int r = e % OR_RC, kk = e / OR_RC;
          Qs[kk * OR_LD + r] = r < nr ? __ldcg(D.Y + (size_t)(r0 + r) + (size_t)kk * D.n) : 0.0;
        }
      } else {
        for (int e = t; e < BS * OR_RC; e += OR_T) {
          const int r = e % OR_RC, jj = e / OR_RC;
          Xn[jj * OR_LD + r] = r < nr ? __ldcg(X + (size_t)(r0 + r) + (size_t)jj * D.n) : 0.0;
        }
      }
      if (q > 0) {
        if (!ready) copy_chunk0(cur, Qs);
        if (cur.s != ss_slot) {
          for (int e = t; e < ke0 * BS; e += OR_T) {
            const int cc = e % ke0, jj = e / ke0;
            Ss[cc * SLD + jj] = cc < kq0 ? __ldcg(D.Sf + (size_t)cc + (size_t)jj * q) : 0.0;
          }
        }
        ss_slot = ke0 >= q ? cur.s : -1;
      }
      cp_async_commit();  // this step's chunk (when not prefetched)
      const bool pre = more && !nxt.skip && J[nxt.s].q > 0;
      if (pre) copy_chunk0(nxt, Qb[qbuf ^ 1]);  // in flight during this step's products
      cp_async_commit();
      cp_async_wait1();   // everything but the group just committed
      __syncthreads();
      ready = pre;
      if (pass && q == 0) {
        for (int e = t; e < BS * OR_RC; e += OR_T) {
          const int r = e % OR_RC, jj = e / OR_RC;
          Xn[jj * OR_LD + r] = r < nr ? xm_entry<BS>(Qs, OR_LD, r, Ms, jj) : 0.0;
        }
      }
      if (q > 0) {
        // each output: two chains (even and odd basis columns) added at the end, so the arithmetic is
        // the same however many rows and basis columns a step stages (zero columns pad a step to even)
        const int nout = nr * BS;
        double ae[MAXO], ao[MAXO];
#pragma unroll
        for (int v = 0; v < MAXO; ++v) ae[v] = ao[v] = 0.0;
        for (int k0 = 0; k0 < q; k0 += kc) {
          const int kq = min(kc, q - k0), ke = (kq + 1) & ~1;
          if (k0 > 0) {
            __syncthreads();
            for (int e = t; e < ke * nr; e += OR_T) {
              const int r = e % nr, cc = e / nr;
              Qs[cc * nr + r] = cc < kq ? D.Q[(size_t)(r0 + r) + (size_t)(k0 + cc) * D.n] : 0.0;
            }
            for (int e = t; e < ke * BS; e += OR_T) {
              const int cc = e % ke, jj = e / ke;
              Ss[cc * SLD + jj] = cc < kq ? __ldcg(D.Sf + (size_t)(k0 + cc) + (size_t)jj * q) : 0.0;
            }
            __syncthreads();
          }
#pragma unroll
          for (int v = 0; v < MAXO; ++v) {
            const int o = t + v * OR_T;
            if (o < nout) {
              const int r = o % nr, jj = o / nr;
#pragma unroll 4
              for (int cc = 0; cc < ke; cc += 2) {
                ae[v] = fma(Qs[cc * nr + r], Ss[cc * SLD + jj], ae[v]);
                ao[v] = fma(Qs[(cc + 1) * nr + r], Ss[(cc + 1) * SLD + jj], ao[v]);
              }
            }
          }
        }
#pragma unroll
        for (int v = 0; v < MAXO; ++v) {
          const int o = t + v * OR_T;
          if (o < nout) Xn[(o / nr) * OR_LD + (o % nr)] -= ae[v] + ao[v];
        }
      }
      __syncthreads();
      if (q > 0 || pass) {  // projected rows (or the rows of W formed here) back in place
        for (int e = t; e < BS * nr; e += OR_T) {
          const int r = e % nr, jj = e / nr;
          X[(size_t)(r0 + r) + (size_t)jj * D.n] = Xn[jj * OR_LD + r];
        }
      }
      for (int b = 0; b < k; ++b) {  // Gram partial of each unit
        const int rb0 = b * RB, rn = min(RB, nr - rb0);
#pragma unroll
        for (int v = 0; v < GE; ++v) {
          const int e = t + v * OR_T;
          if (e < BS * BS) {
            const int a = e % BS, c = e / BS;
            double g = 0.0;
            for (int r = rb0; r < rb0 + rn; ++r) g = fma(Xn[a * OR_LD + r], Xn[c * OR_LD + r], g);
            D.Gp[(size_t)(blk0 + b) * BS * BS + e] = g;
          }
        }
      }
      const int units_in_chunk = min(bpc, D.nrb - rc * bpc);
      if (ticket(D.cnt + D.ncb + rc, k, units_in_chunk)) {
#pragma unroll
        for (int v = 0; v < GE; ++v) {  // the chunk's partial: its units' in order
          const int e = t + v * OR_T;
          if (e < BS * BS) {
            double g = 0.0;
            for (int b = 0; b < units_in_chunk; ++b) g += __ldcg(D.Gp + (size_t)(rc * bpc + b) * BS * BS + e);
            D.Gc[(size_t)rc * BS * BS + e] = g;
          }
        }
        if (ticket(D.cnt + D.ncb + D.nrc, 1, D.nrc)) {
#pragma unroll
          for (int v = 0; v < GE; ++v) {  // G: the chunks' partials in order
            const int e = t + v * OR_T;
            if (e < BS * BS) {
              double g = 0.0;
#pragma unroll 4
              for (int c = 0; c < D.nrc; ++c) g += __ldcg(D.Gc + (size_t)c * BS * BS + e);
              Gs[e] = g;
            }
          }
          __syncthreads();
          if (t < 32) {
            const int nk1 = pass ? __ldcg(D.st + 1) : 0;
            cholqr_slot<BS>(Gs, D.M, D.st, D.en, D.thr, H.tau, pass == 0, nk1);
          }
        }
      }
      qbuf ^= 1;
    } else {
      ready = false;
    }
    if (!more) break;
    u = un;
    cur = nxt;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// out = X M, row-local: pass 0 W = Y M1 (slots with a basis), pass 1 Q[:, q:q+BS] = W M2.  Units of
// OR_T / BS rows; a CTA takes up to a chunk of consecutive units of one slot in one step.
template <int BS>
__device__ void phase_xm(const OrthHdr& H, const OrthDev* J, const int* pd, int total, int pass, double* sm) {
  constexpr int RD = OR_T / BS;
  constexpr int UPC = OR_RC / RD;  // units per chunk
  double* Xs = sm;                 // BS x OR_LD
  double* Ms = sm + BS * OR_LD;    // BS x BS
  const int t = threadIdx.x;
  const Range R = unit_range(pd, H.ns, total);
  int s = R.s, ms_slot = -1;
  for (int u = R.u0; u < R.u1;) {
    s = next_slot(pd, H.ns, s, u);
    const OrthDev& D = J[s];
    const int l0 = u - pd[s], nunits = (D.n + RD - 1) / RD;
    const int k = min(min(R.u1 - u, UPC), nunits - l0);
    u += k;
    if (converged(D)) continue;
    const int r0 = l0 * RD, nr = min(k * RD, D.n - r0);
    const double* X = pass ? D.W : D.Y;
    double* out = pass ? D.Qn : D.W;
    __syncthreads();
    if (s != ms_slot) {
      for (int e = t; e < BS * BS; e += OR_T) Ms[e] = __ldcg(D.M + e);
      ms_slot = s;
    }
    for (int e = t; e < BS * nr; e += OR_T) {
      const int r = e % nr, j = e / nr;
      Xs[j * OR_LD + r] = __ldcg(X + (size_t)(r0 + r) + (size_t)j * D.n);
    }
    __syncthreads();
    for (int e = t; e < BS * nr; e += OR_T) {
      const int r = e % nr, j = e / nr;
      out[(size_t)(r0 + r) + (size_t)j * D.n] = xm_entry<BS>(Xs, OR_LD, r, Ms, j);
    }
  }
}

template <int BS>
__global__ void __launch_bounds__(OR_T) k_orth_round(const char* __restrict__ tab, unsigned* __restrict__ bar) {
  static_assert(OR_T % BS == 0 && OR_RC % (OR_T / BS) == 0, "thread mapping");
  extern __shared__ double sm[];
  const OrthHdr H = *reinterpret_cast<const OrthHdr*>(tab);
  const OrthDev* J = reinterpret_cast<const OrthDev*>(tab + sizeof(OrthHdr));
  const int* pa = reinterpret_cast<const int*>(J + H.ns);
  const int* pb = pa + H.ns + 1;
  const int* pd1 = pb + H.ns + 1;
  const int* pd2 = pd1 + H.ns + 1;
  const bool basis = H.total[0] > 0;
  if (basis) {
    phase_qtx<BS>(H, J, pa, 0, sm);
    if (!grid_sync(bar)) return;
  }
  phase_project<BS>(H, J, pb, 0, sm);
  if (!grid_sync(bar)) return;
  if (basis) {
    phase_xm<BS>(H, J, pd1, H.total[2], 0, sm);
    if (!grid_sync(bar)) return;
    phase_qtx<BS>(H, J, pa, 1, sm);
    if (!grid_sync(bar)) return;
  }
  phase_project<BS>(H, J, pb, 1, sm);
  if (!grid_sync(bar)) return;
  phase_xm<BS>(H, J, pd2, H.total[3], 1, sm);
}

int rows_per_block(int q) { return q == 0 ? 64 : q <= 16 ? 32 : q <= 48 ? 16 : 8; }
int cdiv_i(int a, int b) { return (a + b - 1) / b; }

}  // namespace

bool orth_fused_ok(int bs) { return bs == 16 || bs == 32; }

int orth_timeout_flag(tlr_ctx* ctx) {
  int v = 0;
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  TLR_CUDA(cudaMemcpyFromSymbol(&v, g_orth_timeout, sizeof(int)));
  if (v) {  // tickets and barrier words may be left mid-count: clear them for later launches
    const int zero = 0;
    TLR_CUDA(cudaMemcpyToSymbol(g_orth_timeout, &zero, sizeof(int)));
    for (int l = 0; l < 2; ++l) {
      if (ctx->split_ctr[l]) TLR_CUDA(cudaMemset(ctx->split_ctr[l], 0, ctx->split_ctr_cap[l] * sizeof(int)));
    }
    if (ctx->orth_bar) TLR_CUDA(cudaMemset(ctx->orth_bar, 0, 4 * sizeof(unsigned)));
  }
  return v;
}

namespace {
template <int BS>
void launch_orth(tlr_ctx* ctx, const char* dtab, unsigned* bar) {
  static int per_sm = 0;
  const int smem = or_smem<BS>() * (int)sizeof(double);
  if (!per_sm) {
    if (smem > 48 * 1024)
      TLR_CUDA(cudaFuncSetAttribute(k_orth_round<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int occ = 0;
    TLR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_orth_round<BS>, OR_T, smem));
    TLR_REQUIRE(occ >= 1, TLR_ERR_CUDA, "orthogonalization kernel does not fit an SM");
    per_sm = 1;
  }
  // One CTA per SM: within the resident capacity, so that every CTA reaches the barriers, and the SM
  // keeps room (registers, shared memory) for the side stream's diagonal-tile kernels beside it.
  TLR_SITE_PRE(ctx);
  k_orth_round<BS><<<(unsigned)(per_sm * ctx->sm_count), OR_T, smem, ctx->stream>>>(dtab, bar);
  TLR_LAUNCH_CHECK(ctx);
}
}  // namespace

void orth_round(tlr_ctx* ctx, int bs, const std::vector<OrthSlot>& sl, int* status, double* enorm, double tau,
                Buf& work) {
  const int ns = (int)sl.size();
  if (ns == 0) return;
  TLR_REQUIRE(orth_fused_ok(bs), TLR_ERR_LIMIT, "fused orthogonalization: block width 16 or 32");
  if (!ctx->orth_bar) {
    ctx->orth_bar = static_cast<unsigned*>(dalloc(ctx, 4 * sizeof(unsigned)));
    TLR_CUDA(cudaMemsetAsync(ctx->orth_bar, 0, 4 * sizeof(unsigned), ctx->stream));
  }
  unsigned* bar = ctx->orth_bar + ((ctx->side && ctx->stream == ctx->side) ? 2 : 0);
  // workspace offsets (doubles) and tickets
  const int rd = OR_T / bs;
  std::vector<OrthDev> jd(ns);
  std::vector<int> pa(ns + 1, 0), pb(ns + 1, 0), pd1(ns + 1, 0), pd2(ns + 1, 0);
  size_t wtot = 0, ctot = 0;
  std::vector<size_t> woff(ns), coff(ns);
  for (int s = 0; s < ns; ++s) {
    const OrthSlot& x = sl[s];
    OrthDev& D = jd[s];
    D.n = x.n;
    D.q = x.q;
    D.nrc = cdiv_i(x.n, OR_RC);
    D.ncb = cdiv_i(x.q, OR_CB);
    D.rb = rows_per_block(x.q);
    D.nrb = cdiv_i(x.n, D.rb);
    D.thr = x.thr;
    woff[s] = wtot;
    wtot += (size_t)D.nrc * x.q * bs + (size_t)x.q * bs + (size_t)(D.nrb + D.nrc + 1) * bs * bs;
    wtot = (wtot + 1) & ~size_t(1);
    coff[s] = ctot;
    ctot += D.ncb + D.nrc + 1;
    const int nrd = cdiv_i(x.n, rd);
    pa[s + 1] = pa[s] + (x.q > 0 ? D.ncb * D.nrc : 0);
    pb[s + 1] = pb[s] + D.nrb;
    pd1[s + 1] = pd1[s] + (x.q > 0 ? nrd : 0);
    pd2[s + 1] = pd2[s] + nrd;
  }
  double* w = work.need<double>(std::max<size_t>(wtot, 2));
  int* ctr = split_counters(ctx, ctot);
  for (int s = 0; s < ns; ++s) {
    const OrthSlot& x = sl[s];
    OrthDev& D = jd[s];
    double* p = w + woff[s];
    D.Q = x.Q;
    D.Qn = x.Q + (size_t)x.q * x.n;
    D.Y = x.Y;
    D.W = x.W;
    D.Sp = p;
    p += (size_t)D.nrc * x.q * bs;
    D.Sf = p;
    p += (size_t)x.q * bs;
    D.Gp = p;
    p += (size_t)D.nrb * bs * bs;
    D.Gc = p;
    p += (size_t)D.nrc * bs * bs;
    D.M = p;
    D.cnt = ctr + coff[s];
    D.st = status + 2 * s;
    D.en = enorm + s;
  }
  OrthHdr H{};
  H.ns = ns;
  H.total[0] = pa[ns];
  H.total[1] = pb[ns];
  H.total[2] = pd1[ns];
  H.total[3] = pd2[ns];
  H.tau = tau;
  std::vector<char> tab(sizeof(OrthHdr) + sizeof(OrthDev) * ns + sizeof(int) * 4 * (ns + 1));
  char* h = tab.data();
  memcpy(h, &H, sizeof(H));
  memcpy(h + sizeof(H), jd.data(), sizeof(OrthDev) * ns);
  int* hp = reinterpret_cast<int*>(h + sizeof(H) + sizeof(OrthDev) * ns);
  memcpy(hp, pa.data(), sizeof(int) * (ns + 1));
  memcpy(hp + (ns + 1), pb.data(), sizeof(int) * (ns + 1));
  memcpy(hp + 2 * (ns + 1), pd1.data(), sizeof(int) * (ns + 1));
  memcpy(hp + 3 * (ns + 1), pd2.data(), sizeof(int) * (ns + 1));
  const char* dtab = static_cast<const char*>(upload(ctx, tab.data(), tab.size()));
  double flops = 0;
  for (const OrthSlot& x : sl) flops += 8.0 * x.n * x.q * bs + 6.0 * x.n * bs * bs;
  if (ctx->kprof) kprof_begin(ctx);
  if (bs == 16) launch_orth<16>(ctx, dtab, bar);
  else launch_orth<32>(ctx, dtab, bar);
  if (ctx->kprof) kprof_end(ctx, 7, flops);
}

}  // namespace tlr
