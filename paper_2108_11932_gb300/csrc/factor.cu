// Left-looking TLR Cholesky (Algorithm 6) and LDL^T (Algorithm 10) over a batch of
// independent matrices.
//
// All matrices advance column by column together.  At column k every phase of
// every matrix goes into the same launches:
//   1. Gram factors G_ij = V_ij^T [D_j] V_kj of the column (one batched GEMM),
//   2. on a side stream, overlapped with 3: updateDense D_k = sum_j U_kj G_kj U_kj^T,
//      the dense potrf / LDL^T of A_kk and its inverse (batched over the matrices),
//   3. cholARAUpdate (Algorithm 5): one dynamic ARA batch holding the tiles of every
//      matrix, each round sampling the chains of Equation 2 / 3 (Gram-regrouped),
//   4. the projection (sampleLeftT), batchTrsm as a product with L_kk^{-1}, updateTiles.
// A single matrix is the batch of one.  Each matrix draws its own Gaussian blocks
// (keyed by its seed), and every reduction has a fixed order, so a matrix's result
// does not depend on the other matrices of the batch.
#include <chrono>
#include <cstdio>
#include <memory>
#include <numeric>

#include "internal.h"

namespace tlr {

namespace {

constexpr double U32 = 5.96e-8;  // FP32 unit roundoff, 2^-24

struct Mat {
  explicit Mat(tlr_ctx* c) : G(c), G32(c), E(c), DV(c), DV32(c), Bc(c), Asave(c) {}
  tlr_mat* A = nullptr;  // input, then (on success) the factor
  tlr_mat* F = nullptr;  // factor under construction
  double eps = 0, thr = 0;
  tlr_opts o{};
  int ldl = 0;
  bool mixed = false;
  bool mixed16 = false;  // truncated split products for the samples and projections (TLR_PREC_MIXED)
  tlr_status st = TLR_OK;
  bool live = true;
  int nb = 0, b = 0;
  // column state: this matrix is at column k (matrices of one step may be at different columns)
  int k = 0;
  bool done = false, stepped = false;
  std::chrono::steady_clock::time_point t0;
  int Kk = 0;
  std::vector<int64_t> goff;
  std::vector<int> gld;
  int64_t gtot = 0, R0k = 0, Rk = 0;
  const int* dtab = nullptr;  // device rank/uoff/voff of F (nb x nb each)
  const int64_t* dgoff = nullptr;
  const int* dgld = nullptr;
  int op0 = 0, nops = 0;
  std::vector<int64_t> boff;
  Buf G, G32, E, DV, DV32, Bc;
  Buf Asave;  // TLR_COMP_MODCHOL: the column's updated diagonal tile, kept for Algorithm 8
  int modified = 0;  // diagonal tiles factored by the modified Cholesky
  // TLR_PIVOT_FROBENIUS (Algorithm 9): the diagonal tiles of F hold A(i,i) - D_i for every i >= k (the
  // finished columns' terms are added as each column ends, not by updateDense), and tile rows and
  // columns are exchanged before a step; the compressed input A is rewritten to the exchanged order
  bool piv = false;
  std::vector<float*> AU32, AV32, FU32, FV32;
  std::vector<int64_t> fu32cap;
  // 7-bit chunk planes (int8) of F's U panels relative to 2 (their columns are orthonormal basis
  // vectors, |u| <= 1): 8 planes of b x fuscap[i] each, for the tensor-core split products
  // (b % 16 == 0)
  bool oz = false;
  std::vector<int8_t*> FUs;
  std::vector<int64_t> fuscap;
  // the same planes transposed (row m of Urow_i contiguous along the panel's columns, row stride
  // futcap[i], a multiple of 16; columns past ulen[i] are zero), so that the products with Urow_i
  // as the left operand (Y += Urow_i W_i, B += Urow_k Z) also read it along k
  std::vector<int8_t*> FUt;
  std::vector<int64_t> futcap;
  // slices of F's V panels (written once, at column j) relative to each panel's bound
  std::vector<int8_t*> FVs;
  int* dFVe = nullptr;                 // per panel exponent (device, nb)
  unsigned long long* dFVmax = nullptr;  // per panel largest |v| (device, nb)
  // slices of the compressed input's V panels (static), relative to each panel's bound
  std::vector<int8_t*> AVs;
  int* dAVe = nullptr;
  unsigned long long* dAVmax = nullptr;
  std::vector<double> nA, nL;  // Frobenius norms of the tiles of A and of L (mixed precision rule)
  double fl_exec = 0, fl_model = 0, fl32 = 0;
  int64_t rounds = 0, t32 = 0, t64 = 0;
};

template <typename T>
struct Panels;
template <>
struct Panels<double> {
  static const double* U(const Mat& m, int i) { return m.F->Urow[i]; }
  static const double* AU(const Mat& m, int i) { return m.A->Urow[i]; }
  static const double* AV(const Mat& m, int j) { return m.A->Vcol[j]; }
  static const double* G(const Mat& m) { return static_cast<const double*>(m.G.p); }
};
template <>
struct Panels<float> {
  static const float* U(const Mat& m, int i) { return m.FU32[i]; }
  static const float* AU(const Mat& m, int i) { return m.AU32[i]; }
  static const float* AV(const Mat& m, int j) { return m.AV32[j]; }
  static const float* G(const Mat& m) { return static_cast<const float*>(m.G32.p); }
};

// Sampling chains and projection of column k for the operands (tiles) of all
// matrices of the batch, in arithmetic T (FP64, or FP32 on FP32 copies of the
// panels).  The ARA engine sees FP64 samples.
template <typename T>
struct BatchSampler : Sampler {
  tlr_ctx* ctx = nullptr;
  int bs = 0;
  std::vector<Mat*>* L = nullptr;          // matrices of this column step
  const std::vector<int>* op_m = nullptr;  // operand -> index into L
  const std::vector<int>* op_i = nullptr;  // operand -> tile row i
  const std::vector<char>* member = nullptr;
  const double* Q = nullptr;
  const std::vector<int64_t>* qoff = nullptr;
  Buf *bom = nullptr, *bom32 = nullptr, *bw = nullptr, *by32 = nullptr, *bp = nullptr, *bz = nullptr,
      *bq32 = nullptr, *bb32 = nullptr;
  // tensor-core split products with F's U panels (FP64 arithmetic, matrices with M.oz)
  const int* d_one = nullptr;  // device int 1: the exponent of the U-panel slices
  Buf *bos = nullptr, *boe = nullptr, *bws = nullptr, *bwe = nullptr;  // Omega / W (or Q) slices
  // the compressed input's U0 block of each operand's tile (i, k), sliced once per column step
  // (transposed: rows along its r0 columns, zero-padded to r0w = r0 rounded up to 32), so that
  // Y = [U0 | Urow_i] W is one split product; u0off[op] < 0 where that product stays in FP64 (as for
  // tile-pivoted matrices: a tile moved across the diagonal has the old V0 as its U0, whose entries
  // the slices' fixed bound 2 does not cover)
  Buf* bu0 = nullptr;
  std::vector<int64_t> u0off;
  // the same blocks sliced along their columns (rows along b, like Urow_i's), for P0 = U0^T Q in the
  // projection; u0poff[op] < 0 where that product stays in FP64
  Buf* bu0p = nullptr;
  std::vector<int64_t> u0poff;
  bool u0_ready = false;
  static constexpr bool F32 = sizeof(T) == 4;
  bool owns_omega() const override { return true; }
  bool mine(int op) const { return !member || (*member)[op]; }

  // X and X0 of one matrix for rounds [t0, t1): Kk x bs (t1 - t0) and R0k x bs (t1 - t0), round t's
  // block at column bs (t - t0).  A column's tiles start their ARA at round 0 whenever they enter
  // the batch, so the blocks serve every tile that reaches those rounds.
  struct XRange {
    int t0, t1;
    T* X;
    T* X0;
    std::shared_ptr<Buf> buf;
  };
  std::vector<std::vector<XRange>> xr;  // per matrix of L

  // Forms X = Urow_k^T [Omega_t0 .. Omega_t1-1] (and X0) for the matrices in `ms`, starting at round
  // t: the first range covers the rounds the column's highest-rank tile is expected to need (its
  // compressed rank / bs + 2), a later one half as many.  One Gaussian launch, one slicing and one
  // product of width bs (t1 - t0) replace that many per-round launches; each product keeps the
  // split-K of its one-round shape (rule_n = bs), so every element equals the one-round result.
  void form_ranges(const std::vector<int>& ms, int t) {
    std::vector<int> nr(ms.size());
    std::vector<int64_t> omo(ms.size());
    int64_t omt = 0;
    for (size_t u = 0; u < ms.size(); ++u) {
      const Mat& M = *(*L)[ms[u]];
      int r0max = 0;
      for (int i = M.k + 1; i < M.nb; ++i) r0max = std::max(r0max, M.A->rank[ix(M.A, i, M.k)]);
      int n = (r0max + bs - 1) / bs + 2;
      if (t > 0) n = std::max(2, n / 2);
      const int64_t per = (int64_t)(std::max(M.Kk, 1) + std::max<int64_t>(M.R0k, 1)) * bs * (int64_t)sizeof(T);
      n = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)n, 32, (int64_t)(32 << 20) / per}));
      nr[u] = n;
      omo[u] = omt;
      omt += (int64_t)M.b * bs * n;
    }
    double* Om = bom->need<double>((size_t)omt);
    std::vector<OmegaJob> oj;
    for (size_t u = 0; u < ms.size(); ++u) {
      const Mat& M = *(*L)[ms[u]];
      for (int r = 0; r < nr[u]; ++r)
        oj.push_back(OmegaJob{Om + omo[u] + (size_t)r * M.b * bs, M.o.seed, STREAM_FACTOR, (uint32_t)M.k,
                              (uint32_t)(t + r), M.b, bs});
    }
    omega_batched(ctx, oj);
    const T* OmT = reinterpret_cast<const T*>(Om);
    if (F32) {
      float* o32 = bom32->need<float>((size_t)omt);
      to_float(ctx, omt, Om, o32);
      OmT = reinterpret_cast<const T*>(o32);
    }
    std::vector<GemmJob<T>> jx;
    std::vector<OzColJob> ocj;
    std::vector<OzJob> oxj;
    int64_t ne = 0, nx = 0;
    if (!F32)
      for (size_t u = 0; u < ms.size(); ++u) {
        const Mat& M = *(*L)[ms[u]];
        if (M.oz && (M.Kk > 0 || M.R0k > 0)) { ne += (int64_t)bs * nr[u]; nx += (int64_t)8 * M.b * bs * nr[u]; }
      }
    int8_t* os = bos->need<int8_t>((size_t)std::max<int64_t>(nx, 1));
    int* oe = boe->need<int>((size_t)std::max<int64_t>(ne, 1));
    for (size_t u = 0; u < ms.size(); ++u) {
      Mat& M = *(*L)[ms[u]];
      const int n = nr[u], w = bs * n, kk = std::max(M.Kk, 1), r0k = (int)std::max<int64_t>(M.R0k, 1);
      XRange rg;
      rg.t0 = t;
      rg.t1 = t + n;
      rg.buf = std::make_shared<Buf>(ctx);
      rg.X = rg.buf->template need<T>((size_t)(kk + r0k) * w);
      rg.X0 = rg.X + (size_t)kk * w;
      if (!F32 && M.oz && (M.Kk > 0 || M.R0k > 0)) {
        ocj.push_back(OzColJob{Om + omo[u], os, oe, M.b, w, 0, M.b});
        // X = Urow_k^T Omega: rows of A^T are the panel's columns (k along the b rows)
        if (M.Kk > 0) {
          oxj.push_back(OzJob{M.FUs[M.k], os, d_one, oe, reinterpret_cast<double*>(rg.X),
                              (size_t)M.b * M.fuscap[M.k], (size_t)M.b * w, M.b, M.Kk, M.Kk, w, M.b});
          oxj.back().rule_n = bs;
        }
        // X0 = V0col_k^T Omega with the slices of the compressed input's V panel
        if (M.R0k > 0) {
          oxj.push_back(OzJob{M.AVs[M.k], os, M.dAVe + M.k, oe, reinterpret_cast<double*>(rg.X0),
                              (size_t)M.b * M.R0k, (size_t)M.b * w, M.b, (int)M.R0k, (int)M.R0k, w, M.b});
          oxj.back().rule_n = bs;
        }
        os += (size_t)8 * M.b * w;
        oe += w;
      } else {
        if (M.Kk > 0) {
          jx.push_back(job<T>(TN, M.Kk, w, Panels<T>::U(M, M.k), M.b, OmT + omo[u], M.b, M.b, rg.X, M.Kk, 1.0, 0.0));
          jx.back().rule_n = bs;
        }
        if (M.R0k > 0) {
          jx.push_back(job<T>(TN, (int)M.R0k, w, Panels<T>::AV(M, M.k), M.b, OmT + omo[u], M.b, M.b, rg.X0,
                              (int)M.R0k, 1.0, 0.0));
          jx.back().rule_n = bs;
        }
      }
      (F32 ? M.fl32 : M.fl_exec) += 2.0 * M.b * w * (M.Kk + M.R0k);
      xr[ms[u]].push_back(std::move(rg));
    }
    gemm<T>(ctx, TN, jx);
    oz_split_cols(ctx, ocj);
    oz_gemm(ctx, oxj);
  }

  static int round32(int r) { return (r + 31) / 32 * 32; }
  void prepare_u0() {
    u0_ready = true;
    const int nops = (int)op_m->size();
    u0off.assign(nops, -1);
    u0poff.assign(nops, -1);
    if (F32 || !bu0 || !bu0p) return;
    {  // column-oriented slices for the projection
      int64_t tot = 0;
      for (int op = 0; op < nops; ++op) {
        if (!mine(op)) continue;
        const Mat& M = *(*L)[(*op_m)[op]];
        const int i = (*op_i)[op], r0 = M.A->rank[ix(M.A, i, M.k)];
        if (!M.oz || r0 == 0 || M.piv) continue;
        u0poff[op] = tot;
        tot += (int64_t)8 * M.b * r0;
      }
      if (tot > 0) {
        int8_t* base = bu0p->need<int8_t>((size_t)tot);
        std::vector<OzColJob> cj;
        for (int op = 0; op < nops; ++op) {
          if (u0poff[op] < 0) continue;
          const Mat& M = *(*L)[(*op_m)[op]];
          const int i = (*op_i)[op], r0 = M.A->rank[ix(M.A, i, M.k)];
          OzColJob c{reinterpret_cast<const double*>(Panels<T>::AU(M, i)) + (size_t)M.b * M.A->uoff[ix(M.A, i, M.k)],
                     base + u0poff[op], nullptr, M.b, r0, 0, M.b};
          c.efix = 1;
          cj.push_back(c);
        }
        oz_split_cols(ctx, cj);
      }
    }
    int64_t tot = 0;
    for (int op = 0; op < nops; ++op) {
      if (!mine(op)) continue;
      const Mat& M = *(*L)[(*op_m)[op]];
      const int i = (*op_i)[op], r0 = M.A->rank[ix(M.A, i, M.k)];
      if (!M.oz || r0 == 0 || M.piv || round32(r0) + M.F->ulen[i] > 16384) continue;
      u0off[op] = tot;
      tot += (int64_t)8 * M.b * round32(r0);
    }
    if (tot == 0) return;
    int8_t* base = bu0->need<int8_t>((size_t)tot);
    TLR_CUDA(cudaMemsetAsync(base, 0, (size_t)tot, ctx->stream));
    std::vector<OzColJob> cj;
    for (int op = 0; op < nops; ++op) {
      if (u0off[op] < 0) continue;
      const Mat& M = *(*L)[(*op_m)[op]];
      const int i = (*op_i)[op], r0 = M.A->rank[ix(M.A, i, M.k)], r0w = round32(r0);
      OzColJob c{reinterpret_cast<const double*>(Panels<T>::AU(M, i)) + (size_t)M.b * M.A->uoff[ix(M.A, i, M.k)],
                 base + u0off[op], nullptr, M.b, r0, 0, M.b};
      c.plane = (size_t)M.b * r0w;
      c.efix = 1;
      c.tld = r0w;
      cj.push_back(c);
    }
    oz_split_cols(ctx, cj);
  }

  void sample(const std::vector<int>& ops, int t, const double*, const std::vector<double*>& Ydst) override {
    if (!u0_ready) prepare_u0();
    // matrices present in this call
    std::vector<int> mp;
    std::vector<int> slot_of_m(L->size(), -1);
    for (int op : ops) {
      const int m = (*op_m)[op];
      if (slot_of_m[m] < 0) { slot_of_m[m] = (int)mp.size(); mp.push_back(m); }
    }
    // the shared products X = Urow_k^T Omega_t and X0 = V0col_k^T Omega_t of each matrix, formed for a
    // range of rounds at once
    if (xr.size() < L->size()) xr.resize(L->size());
    std::vector<const XRange*> rng(mp.size(), nullptr);
    std::vector<int> need;
    for (size_t u = 0; u < mp.size(); ++u) {
      for (const auto& r : xr[mp[u]])
        if (t >= r.t0 && t < r.t1) rng[u] = &r;
      if (!rng[u]) need.push_back(mp[u]);
    }
    if (!need.empty()) {
      form_ranges(need, t);
      for (size_t u = 0; u < mp.size(); ++u)
        if (!rng[u]) rng[u] = &xr[mp[u]].back();
    }
    // W blocks of every operand (block-diagonal Gram products), then Y = [U0 | Urow] W
    std::vector<SlotDescT<T>> sd(ops.size());
    int64_t wtot = 0, ytot = 0;
    for (size_t s = 0; s < ops.size(); ++s) {
      const int op = ops[s], u = slot_of_m[(*op_m)[op]], i = (*op_i)[op];
      const Mat& M = *(*L)[(*op_m)[op]];
      SlotDescT<T>& d = sd[s];
      d.rank = M.dtab;
      d.uoff = M.dtab + (size_t)M.nb * M.nb;
      d.voff = M.dtab + (size_t)2 * M.nb * M.nb;
      d.goff = M.dgoff;
      d.gld = M.dgld;
      d.G = Panels<T>::G(M);
      d.ldx = std::max(M.Kk, 1);
      d.ldx0 = (int)std::max<int64_t>(M.R0k, 1);
      d.X = rng[u]->X + (size_t)d.ldx * bs * (t - rng[u]->t0);
      d.X0 = rng[u]->X0 + (size_t)d.ldx0 * bs * (t - rng[u]->t0);
      d.nb = M.nb;
      d.k = M.k;
      d.i = i;
      d.r0 = M.A->rank[ix(M.A, i, M.k)];
      d.x0off = (int)M.A->voff[ix(M.A, i, M.k)];
      d.Ki = (int)M.F->ulen[i];
      d.Kk = M.Kk;
      d.q = bs;
      d.bs = bs;
      d.r0w = u0off[op] >= 0 ? round32(d.r0) : d.r0;
      d.W = reinterpret_cast<T*>(wtot);  // offset, fixed below
      d.P = nullptr;
      d.Z = nullptr;
      wtot += (int64_t)(d.r0w + d.Ki) * bs;
      ytot += (int64_t)M.b * bs;
    }
    T* W = bw->need<T>((size_t)std::max<int64_t>(wtot, 1));
    for (auto& d : sd) d.W = W + reinterpret_cast<size_t>(d.W);
    const SlotDescT<T>* sdd = static_cast<const SlotDescT<T>*>(upload(ctx, sd.data(), sd.size() * sizeof(SlotDescT<T>)));
    std::vector<BlkItem> items;
    for (size_t s = 0; s < ops.size(); ++s) {  // -G_ij X_j: r_ij x bs tiles; the X0 copy: r0 x bs
      const Mat& M = *(*L)[(*op_m)[ops[s]]];
      const int i = sd[s].i;
      for (int j = 0; j <= M.k; ++j) {
        const int R = j < M.k ? M.F->rank[ix(M.F, i, j)] : sd[s].r0w;
        for (int rc = 0; 16 * rc < R; ++rc)
          for (int cc = 0; 16 * cc < bs; ++cc)
            items.push_back(BlkItem{(uint32_t)s, (uint16_t)j, (uint8_t)rc, (uint8_t)cc});
      }
    }
    blkdiag_sample<T>(ctx, items, sdd);
    T* Y32 = F32 ? reinterpret_cast<T*>(by32->need<float>((size_t)ytot)) : nullptr;
    std::vector<GemmJob<T>> jy;
    std::vector<ConvBackJob> cb;
    std::vector<OzColJob> wcj;
    std::vector<OzJob> wyj;
    int64_t yo = 0;
    // split path: Y = [U0 | Urow_i] W as one product when U0 has slices (K = r0w + Ki), or Urow_i W_i
    // after the FP64 product with U0 when it has none
    auto folded = [&](size_t s) { return u0off[ops[s]] >= 0; };
    auto split_k = [&](size_t s) -> int {
      const Mat& M = *(*L)[(*op_m)[ops[s]]];
      if (F32 || !M.oz) return 0;
      if (folded(s)) return sd[s].r0w + sd[s].Ki;
      return (sd[s].Ki > 0 && sd[s].Ki <= 16384) ? sd[s].Ki : 0;
    };
    int64_t wsl = 0, wex = 0;  // slices of the W_i rows of the split products
    for (size_t s = 0; s < ops.size(); ++s) {
      const int ks = split_k(s);
      if (ks > 0) { wsl += (int64_t)8 * oz_ld(ks) * bs; wex += bs; }
    }
    int8_t* ws_ = wsl ? bws->need<int8_t>((size_t)wsl) : nullptr;
    int* we_ = wex ? bwe->need<int>((size_t)wex) : nullptr;
    for (size_t s = 0; s < ops.size(); ++s) {
      const int op = ops[s], i = (*op_i)[op];
      Mat& M = *(*L)[(*op_m)[op]];
      const int r0 = sd[s].r0, r0w = sd[s].r0w, Ki = sd[s].Ki, ldw = std::max(r0w + Ki, 1);
      T* Yo = F32 ? Y32 + yo : reinterpret_cast<T*>(Ydst[s]);
      const T* U0 = r0 ? Panels<T>::AU(M, i) + (size_t)M.b * M.A->uoff[ix(M.A, i, M.k)] : nullptr;
      GemmJob<T> g = job<T>(NN, M.b, bs, U0, M.b, sd[s].W, ldw, r0, Yo, M.b, 1.0, 0.0);
      const int ks = split_k(s);  // exact integer totals need K <= 16384
      if (ks > 0) {
        const int ldo = oz_ld(ks);
        const int w0 = folded(s) ? 0 : r0;  // first W row of the product
        OzColJob c{reinterpret_cast<const double*>(sd[s].W + w0), ws_, we_, ldw, bs, 0, ks};
        c.ldo = ldo;
        wcj.push_back(c);
        OzJob y{M.FUt[i], ws_, d_one, we_, reinterpret_cast<double*>(Yo), (size_t)M.b * M.futcap[i],
                (size_t)ldo * bs, (int)M.futcap[i], M.b, M.b, bs, ks};
        y.ldb = ldo;
        if (folded(s)) {  // Y = [U0 | Urow_i] W on the tensor cores alone
          const int8_t* u0 = static_cast<const int8_t*>(bu0->p) + u0off[ops[s]];
          if (Ki > 0) {
            y.A0 = u0;
            y.sA0 = (size_t)M.b * r0w;
            y.lda0 = r0w;
            y.K0 = r0w;
          } else {
            y.A = u0;
            y.sA = (size_t)M.b * r0w;
            y.lda = r0w;
          }
          y.accumulate = 0;
        } else {  // Y = U0 W[0:r0] in FP64 first, then + Urow_i W[r0:]
          y.accumulate = 1;
          jy.push_back(g);
        }
        if (M.mixed16) y.tol = M.thr / (8.0 * std::sqrt((double)M.b));  // column norm of Y within thr / 8
        wyj.push_back(y);
        ws_ += (size_t)8 * ldo * bs;
        we_ += bs;
      } else {
        g.A[1] = Panels<T>::U(M, i);
        g.lda[1] = M.b;
        g.B[1] = sd[s].W + r0;
        g.ldb[1] = ldw;
        g.K[1] = Ki;
        jy.push_back(g);
      }
      if (F32) cb.push_back(ConvBackJob{reinterpret_cast<const float*>(Yo), Ydst[s], (int64_t)M.b * bs});
      yo += (int64_t)M.b * bs;
      (F32 ? M.fl32 : M.fl_exec) += 2.0 * M.b * bs * (r0 + Ki);
      double R = r0;  // paper model: 4 products per (i, j) pair, Equation 2
      for (int j = 0; j < M.k; ++j) R += M.F->rank[ix(M.F, i, j)] + M.F->rank[ix(M.F, M.k, j)];
      M.fl_model += 4.0 * M.b * bs * R;
      (F32 ? M.t32 : M.t64) += 1;
    }
    gemm<T>(ctx, NN, jy);
    oz_split_cols(ctx, wcj);
    oz_gemm(ctx, wyj);
    batched_to_double(ctx, cb);
  }

  void project(const std::vector<int>& q) override {
    const int nops = (int)q.size();
    std::vector<int> ops;
    for (int op = 0; op < nops; ++op)
      if (mine(op) && q[op] > 0) ops.push_back(op);
    if (ops.empty()) return;
    std::vector<SlotDescT<T>> sd(ops.size());
    int64_t ptot = 0, ztot = 0, q32tot = 0;
    std::vector<int64_t> q32o(ops.size());
    for (size_t s = 0; s < ops.size(); ++s) {
      const int op = ops[s], i = (*op_i)[op];
      const Mat& M = *(*L)[(*op_m)[op]];
      SlotDescT<T>& d = sd[s];
      d.rank = M.dtab;
      d.uoff = M.dtab + (size_t)M.nb * M.nb;
      d.voff = M.dtab + (size_t)2 * M.nb * M.nb;
      d.goff = M.dgoff;
      d.gld = M.dgld;
      d.G = Panels<T>::G(M);
      d.nb = M.nb;
      d.k = M.k;
      d.i = i;
      d.r0 = M.A->rank[ix(M.A, i, M.k)];
      d.Ki = (int)M.F->ulen[i];
      d.Kk = M.Kk;
      d.q = q[op];
      d.bs = bs;
      d.P = reinterpret_cast<T*>(ptot);
      d.Z = reinterpret_cast<T*>(ztot);
      ptot += (int64_t)(d.r0 + d.Ki) * q[op];
      ztot += (int64_t)(d.r0 + M.Kk) * q[op];
      q32o[s] = q32tot;
      q32tot += (int64_t)M.b * q[op];
    }
    T* P = bp->need<T>((size_t)std::max<int64_t>(ptot, 1));
    T* Z = bz->need<T>((size_t)std::max<int64_t>(ztot, 1));
    for (auto& d : sd) {
      d.P = P + reinterpret_cast<size_t>(d.P);
      d.Z = Z + reinterpret_cast<size_t>(d.Z);
    }
    // Q_i and the output B_i in arithmetic T
    float* Q32 = nullptr;
    float* B32 = nullptr;
    if (F32) {
      Q32 = bq32->need<float>((size_t)std::max<int64_t>(q32tot, 1));
      B32 = bb32->need<float>((size_t)std::max<int64_t>(q32tot, 1));
      std::vector<ConvJob> cj;
      for (size_t s = 0; s < ops.size(); ++s) {
        const int op = ops[s];
        const Mat& M = *(*L)[(*op_m)[op]];
        cj.push_back(ConvJob{Q + (*qoff)[op], Q32 + q32o[s], (int64_t)M.b * q[op]});
      }
      batched_to_float(ctx, cj);
    }
    auto Qop = [&](size_t s) -> const T* {
      return F32 ? reinterpret_cast<const T*>(Q32 + q32o[s]) : reinterpret_cast<const T*>(Q + (*qoff)[ops[s]]);
    };
    std::vector<GemmJob<T>> jp;
    std::vector<OzColJob> qcj;
    std::vector<OzJob> pqj;
    if (!u0_ready) prepare_u0();
    auto p0_split = [&](size_t s) { return !F32 && u0poff[ops[s]] >= 0; };
    int64_t qsl = 0, qex = 0;  // slices of Q_i for the split products with Urow_i and U0
    if (!F32)
      for (size_t s = 0; s < ops.size(); ++s) {
        const Mat& M = *(*L)[(*op_m)[ops[s]]];
        if (M.oz && (sd[s].Ki > 0 || p0_split(s))) { qsl += (int64_t)8 * M.b * q[ops[s]]; qex += q[ops[s]]; }
      }
    int8_t* qs_ = qsl ? bws->need<int8_t>((size_t)qsl) : nullptr;
    int* qe_ = qex ? bwe->need<int>((size_t)qex) : nullptr;
    for (size_t s = 0; s < ops.size(); ++s) {
      const int op = ops[s], i = (*op_i)[op];
      Mat& M = *(*L)[(*op_m)[op]];
      const int r0 = sd[s].r0, Ki = sd[s].Ki, ldp = r0 + Ki;
      const bool qsplit = !F32 && M.oz && (Ki > 0 || p0_split(s));
      if (qsplit) qcj.push_back(OzColJob{reinterpret_cast<const double*>(Qop(s)), qs_, qe_, M.b, q[op], 0, M.b});
      if (r0 > 0) {
        if (p0_split(s)) {  // P[0:r0] = U0^T Q_i on the tensor cores
          pqj.push_back(OzJob{static_cast<const int8_t*>(bu0p->p) + u0poff[op], qs_, d_one, qe_,
                              reinterpret_cast<double*>(sd[s].P), (size_t)M.b * r0, (size_t)M.b * q[op], M.b, ldp,
                              r0, q[op], M.b});
        } else {
          jp.push_back(job<T>(TN, r0, q[op], Panels<T>::AU(M, i) + (size_t)M.b * M.A->uoff[ix(M.A, i, M.k)], M.b,
                              Qop(s), M.b, M.b, sd[s].P, ldp, 1.0, 0.0));
        }
      }
      if (Ki > 0) {
        if (!F32 && M.oz) {  // P[r0:] = Urow_i^T Q_i on the tensor cores
          pqj.push_back(OzJob{M.FUs[i], qs_, d_one, qe_, reinterpret_cast<double*>(sd[s].P + r0),
                              (size_t)M.b * M.fuscap[i], (size_t)M.b * q[op], M.b, ldp, Ki, q[op], M.b});
        } else {
          jp.push_back(job<T>(TN, Ki, q[op], Panels<T>::U(M, i), M.b, Qop(s), M.b, M.b, sd[s].P + r0, ldp, 1.0, 0.0));
        }
      }
      if (qsplit) {
        qs_ += (size_t)8 * M.b * q[op];
        qe_ += q[op];
      }
      (F32 ? M.fl32 : M.fl_exec) += 2.0 * M.b * q[op] * (r0 + Ki);
    }
    gemm<T>(ctx, TN, jp);
    oz_split_cols(ctx, qcj);
    oz_gemm(ctx, pqj);
    const SlotDescT<T>* sdd = static_cast<const SlotDescT<T>*>(upload(ctx, sd.data(), sd.size() * sizeof(SlotDescT<T>)));
    std::vector<BlkItem> items;
    for (size_t s = 0; s < ops.size(); ++s) {  // -G_ij^T P_j: r_kj x q tiles; the P0 copy: r0 x q
      const Mat& M = *(*L)[(*op_m)[ops[s]]];
      for (int j = 0; j <= M.k; ++j) {
        const int R = j < M.k ? M.F->rank[ix(M.F, M.k, j)] : sd[s].r0;
        for (int rc = 0; 16 * rc < R; ++rc)
          for (int cc = 0; 16 * cc < sd[s].q; ++cc)
            items.push_back(BlkItem{(uint32_t)s, (uint16_t)j, (uint8_t)rc, (uint8_t)cc});
      }
    }
    blkdiag_project<T>(ctx, items, sdd);
    std::vector<GemmJob<T>> jb;
    std::vector<ConvBackJob> cb;
    std::vector<OzColJob> zcj;
    std::vector<OzJob> zbj;
    int64_t zsl = 0, zex = 0;  // slices of the Z_i rows that multiply Urow_k (split path)
    if (!F32)
      for (size_t s = 0; s < ops.size(); ++s) {
        const Mat& M = *(*L)[(*op_m)[ops[s]]];
        if (M.oz && M.Kk > 0 && M.Kk <= 16384) { zsl += (int64_t)8 * oz_ld(M.Kk) * q[ops[s]]; zex += q[ops[s]]; }
      }
    int8_t* zs_ = zsl ? bws->need<int8_t>((size_t)zsl) : nullptr;
    int* ze_ = zex ? bwe->need<int>((size_t)zex) : nullptr;
    for (size_t s = 0; s < ops.size(); ++s) {
      const int op = ops[s], i = (*op_i)[op];
      Mat& M = *(*L)[(*op_m)[op]];
      const int r0 = sd[s].r0, ldz = std::max(r0 + M.Kk, 1);
      double* Bdst = static_cast<double*>(M.Bc.p) + (size_t)M.boff[op - M.op0] * M.b;
      T* Bo = F32 ? reinterpret_cast<T*>(B32 + q32o[s]) : reinterpret_cast<T*>(Bdst);
      const T* V0 = r0 ? Panels<T>::AV(M, M.k) + (size_t)M.b * M.A->voff[ix(M.A, i, M.k)] : nullptr;
      GemmJob<T> g = job<T>(NN, M.b, q[op], V0, M.b, sd[s].Z, ldz, r0, Bo, M.b, 1.0, 0.0);
      if (!F32 && M.oz && M.Kk > 0 && M.Kk <= 16384) {  // B = V0 Z[0:r0] here, + Urow_k Z[r0:] split
        const int ldo = oz_ld(M.Kk);
        OzColJob c{reinterpret_cast<const double*>(sd[s].Z + r0), zs_, ze_, ldz, q[op], 0, M.Kk};
        c.ldo = ldo;
        zcj.push_back(c);
        OzJob bj{M.FUt[M.k], zs_, d_one, ze_, reinterpret_cast<double*>(Bo), (size_t)M.b * M.futcap[M.k],
                 (size_t)ldo * q[op], (int)M.futcap[M.k], M.b, M.b, q[op], M.Kk};
        bj.ldb = ldo;
        bj.accumulate = 1;
        // the projection B_i = A(i,k)^T Q_i within thr / 8 in Frobenius norm (it enters the tile as Q B^T)
        if (M.mixed16) bj.tol = M.thr / (8.0 * std::sqrt((double)M.b * q[op]));
        zbj.push_back(bj);
        zs_ += (size_t)8 * ldo * q[op];
        ze_ += q[op];
      } else {
        g.A[1] = Panels<T>::U(M, M.k);
        g.lda[1] = M.b;
        g.B[1] = sd[s].Z + r0;
        g.ldb[1] = ldz;
        g.K[1] = M.Kk;
      }
      jb.push_back(g);
      if (F32) cb.push_back(ConvBackJob{reinterpret_cast<const float*>(Bo), Bdst, (int64_t)M.b * q[op]});
      (F32 ? M.fl32 : M.fl_exec) += 2.0 * M.b * q[op] * (r0 + M.Kk);
      double R = r0;
      for (int j = 0; j < M.k; ++j) R += M.F->rank[ix(M.F, i, j)] + M.F->rank[ix(M.F, M.k, j)];
      M.fl_model += 4.0 * M.b * q[op] * R;
    }
    gemm<T>(ctx, NN, jb);
    oz_split_cols(ctx, zcj);
    oz_gemm(ctx, zbj);
    batched_to_double(ctx, cb);
  }
};

// Operands split by the per-tile precision rule; both precisions share the slot layout.
struct SplitSampler : Sampler {
  BatchSampler<double>* f64;
  BatchSampler<float>* f32;
  const std::vector<char>* is32;
  bool owns_omega() const override { return true; }
  void sample(const std::vector<int>& ops, int t, const double* Om, const std::vector<double*>& Y) override {
    std::vector<int> o32, o64;
    std::vector<double*> y32, y64;
    for (size_t s = 0; s < ops.size(); ++s) {
      if ((*is32)[ops[s]]) { o32.push_back(ops[s]); y32.push_back(Y[s]); }
      else { o64.push_back(ops[s]); y64.push_back(Y[s]); }
    }
    if (!o32.empty()) f32->sample(o32, t, Om, y32);
    if (!o64.empty()) f64->sample(o64, t, Om, y64);
  }
  void project(const std::vector<int>& q) override {
    f32->project(q);
    f64->project(q);
  }
};

float* f32_alloc(tlr_ctx* ctx, int64_t n) {
  return static_cast<float*>(dalloc(ctx, sizeof(float) * (size_t)std::max<int64_t>(n, 1)));
}

// Frobenius norms of the tiles of block column j (|V_ij|_F = |U_ij V_ij^T|_F, U orthonormal).
void panel_tile_norms(tlr_ctx* ctx, const tlr_mat* M, int j, std::vector<double>& out, Buf& tmp) {
  const int64_t n = M->vlen[j];
  if (n == 0) return;
  double* d = tmp.need<double>((size_t)n);
  col_sqnorms(ctx, M->Vcol[j], M->b, n, d);
  std::vector<double> h(n);
  TLR_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int i = j + 1; i < M->nb; ++i) {
    double sq = 0;
    for (int c = 0; c < M->rank[ix(M, i, j)]; ++c) sq += h[M->voff[ix(M, i, j)] + c];
    out[ix(M, i, j)] = std::sqrt(sq);
  }
}

void free_f32(tlr_ctx* ctx, Mat& M) {
  for (Buf* bf : {&M.G, &M.G32, &M.E, &M.DV, &M.DV32, &M.Bc}) bf->release();  // per-matrix work buffers
  for (auto* v : {&M.AU32, &M.AV32, &M.FU32, &M.FV32})
    for (float*& p : *v) {
      dfree(ctx, p);
      p = nullptr;
    }
  for (auto* v : {&M.FUs, &M.FUt, &M.FVs, &M.AVs})
    for (int8_t*& p : *v) {
      dfree(ctx, p);
      p = nullptr;
    }
  for (int** p : {&M.dFVe, &M.dAVe}) {
    dfree(ctx, *p);
    *p = nullptr;
  }
  for (unsigned long long** p : {&M.dFVmax, &M.dAVmax}) {
    dfree(ctx, *p);
    *p = nullptr;
  }
}

}  // namespace

// A set of factorizations in flight: matrices join with add(), every step() advances
// each unfinished matrix by one column (each at its own column index), finished
// matrices leave.  factor_batch is add() of all matrices then step() until done;
// the serving loop adds requests between steps (continuous batching).
struct Session {
  tlr_ctx* ctx;
  int bs = -1;
  std::vector<std::unique_ptr<Mat>> mats;
  Buf bnrm, bQ, bTab, bInfo, bTmp, bTmpMain, bOm, bOm32, bW, bY32, bP, bZ, bQ32, bB32;
  Buf bOzMax, bOzS, bOzE, bOzX, bOzEx;  // split trsm products
  Buf bOzOs, bOzOe, bOzWs, bOzWe, bOne;  // split sampling / projection products
  Buf bOzDs, bOzDe, bOzDm;               // split updateDense products (side stream)
  Buf bMcW, bMcT;                        // modified Cholesky workspaces (main stream)
  Buf bOzU0, bOzU0p;                     // slices of the column's U0 blocks (split sampling / projection)
  Buf bPiv, bPivG, bPivE, bSwap, bSwapV;  // tile pivoting: norms, dense-update products, exchange staging
  Buf bPivS, bPivX;                       // tile pivoting: chunk planes and bounds of the dense updates
  int* d_one = nullptr;
  AraStats total;
  explicit Session(tlr_ctx* c)
      : ctx(c), bnrm(c), bQ(c), bTab(c), bInfo(c), bTmp(c), bTmpMain(c), bOm(c), bOm32(c), bW(c), bY32(c), bP(c), bZ(c),
        bQ32(c), bB32(c), bOzMax(c), bOzS(c), bOzE(c), bOzX(c), bOzEx(c), bOzOs(c), bOzOe(c), bOzWs(c), bOzWe(c),
        bOne(c), bOzDs(c), bOzDe(c), bOzDm(c), bMcW(c), bMcT(c), bOzU0(c), bOzU0p(c), bPiv(c), bPivG(c), bPivE(c),
        bSwap(c), bSwapV(c), bPivS(c), bPivX(c) {
    static const int one = 1;
    d_one = bOne.need<int>(1);
    TLR_CUDA(cudaMemcpyAsync(d_one, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  ~Session() {
    cudaStreamSynchronize(ctx->side);
    cudaStreamSynchronize(ctx->main);
    for (auto& M : mats) {
      free_f32(ctx, *M);
      if (M->F) mat_destroy(ctx, M->F);
    }
  }
  bool busy() const {
    for (auto& M : mats)
      if (M->live && !M->done) return true;
    return false;
  }

  int add(tlr_mat* A, double eps, const tlr_opts& o, int ldl) {
    if (bs < 0) bs = o.bs;
    TLR_REQUIRE(o.bs == bs, TLR_ERR_ARG, "all matrices of a batch use one ARA block width");
    mats.emplace_back(new Mat(ctx));
    Mat& M = *mats.back();
    M.t0 = std::chrono::steady_clock::now();
    M.A = A;
    M.eps = eps;
    M.thr = eps / HALKO;
    M.o = o;
    M.ldl = ldl;
    M.nb = A->nb;
    M.b = A->b;
    M.k = 0;
    M.mixed = o.precision == TLR_PREC_FP32 && eps >= 1e-4;
    M.mixed16 = o.precision == TLR_PREC_MIXED && eps >= 1e-4;
    const int nb = M.nb, b = M.b;
    tlr_mat* F = mat_new(A->N, A->d, b);
    M.F = F;
    F->kern = A->kern;
    F->eps = eps;
    F->diag = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b * b));
    TLR_CUDA(cudaMemcpyAsync(F->diag, A->diag, sizeof(double) * (size_t)nb * b * b, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    if (ldl) F->dvec = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b));
    F->dinv = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)nb * b * b));
    M.piv = o.pivot == TLR_PIVOT_FROBENIUS;
    if (M.piv && o.compensation == TLR_COMP_SHIFT && o.shift != 0.0) {  // A + shift I, before any selection
      std::vector<DiagJob> dj;
      for (int i = 0; i < nb; ++i) dj.push_back(DiagJob{F->diag + (size_t)i * b * b, b, b, o.shift});
      batched_add_diag(ctx, dj);
    }
    for (int i = 0; i < nb; ++i) ensure_ucap(ctx, F, i, std::max<int64_t>(A->ulen[i], 16));
    M.oz = b % 16 == 0;
    if (M.oz) {
      M.FUs.assign(nb, nullptr);
      M.fuscap.assign(nb, 0);
      M.FUt.assign(nb, nullptr);
      M.futcap.assign(nb, 0);
      for (int i = 0; i < nb; ++i) {
        M.fuscap[i] = F->ucap[i];
        M.FUs[i] = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * M.fuscap[i]));
        M.futcap[i] = oz_ld((int)F->ucap[i]);
        M.FUt[i] = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * M.futcap[i]));
        TLR_CUDA(cudaMemsetAsync(M.FUt[i], 0, 8 * (size_t)b * M.futcap[i], ctx->stream));
      }
      M.FVs.assign(nb, nullptr);
      M.dFVe = static_cast<int*>(dalloc(ctx, sizeof(int) * nb));
      M.dFVmax = static_cast<unsigned long long*>(dalloc(ctx, sizeof(unsigned long long) * nb));
      M.AVs.assign(nb, nullptr);
      M.dAVe = static_cast<int*>(dalloc(ctx, sizeof(int) * nb));
      M.dAVmax = static_cast<unsigned long long*>(dalloc(ctx, sizeof(unsigned long long) * nb));
      std::vector<OzColJob> vcj;
      for (int j = 0; j < nb; ++j) {
        if (A->vlen[j] == 0) continue;
        M.AVs[j] = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * A->vlen[j]));
        oz_absmax(ctx, 1, (int64_t)b * A->vlen[j], A->Vcol[j], M.dAVmax + j);
        OzColJob c{A->Vcol[j], M.AVs[j], M.dAVe + j, b, (int)A->vlen[j], 0, b};
        c.emax = M.dAVmax + j;
        vcj.push_back(c);
      }
      oz_split_cols(ctx, vcj);
    }
    if (M.mixed) {  // FP32 copies of A's panels; tile norms for the precision rule
      M.AU32.assign(nb, nullptr);
      M.AV32.assign(nb, nullptr);
      M.FU32.assign(nb, nullptr);
      M.FV32.assign(nb, nullptr);
      M.fu32cap.assign(nb, 0);
      std::vector<ConvJob> cj;
      for (int i = 0; i < nb; ++i) {
        M.AU32[i] = f32_alloc(ctx, (int64_t)b * A->ulen[i]);
        M.AV32[i] = f32_alloc(ctx, (int64_t)b * A->vlen[i]);
        cj.push_back(ConvJob{A->Urow[i], M.AU32[i], (int64_t)b * A->ulen[i]});
        cj.push_back(ConvJob{A->Vcol[i], M.AV32[i], (int64_t)b * A->vlen[i]});
        M.fu32cap[i] = F->ucap[i];
        M.FU32[i] = f32_alloc(ctx, (int64_t)b * M.fu32cap[i]);
      }
      batched_to_float(ctx, cj);
      M.nA.assign((size_t)nb * nb, 0.0);
      M.nL.assign((size_t)nb * nb, 0.0);
      for (int j = 0; j < nb; ++j) panel_tile_norms(ctx, A, j, M.nA, bnrm);
    }
    return (int)mats.size() - 1;
  }

  tlr_status status(int idx) const { return mats[idx]->st; }
  bool finished(int idx) const { return mats[idx]->done || !mats[idx]->live; }

  // A := its factor (the matrix finished its last column).
  void finalize(Mat& M) {
    TLR_CUDA(cudaStreamSynchronize(ctx->main));
    free_f32(ctx, M);
    tlr_mat* A = M.A;
    tlr_mat* F = M.F;
    const int nb = M.nb;
    mat_free_storage(ctx, A);
    dfree(ctx, A->diag);
    dfree(ctx, A->dvec);
    dfree(ctx, A->dinv);
    A->diag = F->diag; F->diag = nullptr;
    A->dvec = F->dvec; F->dvec = nullptr;
    A->dinv = F->dinv; F->dinv = nullptr;
    A->rank = F->rank; A->uoff = F->uoff; A->voff = F->voff;
    A->Urow = F->Urow; A->Vcol = F->Vcol; A->ucap = F->ucap; A->vlen = F->vlen; A->ulen = F->ulen;
    F->Urow.assign(nb, nullptr);
    F->Vcol.assign(nb, nullptr);
    mat_destroy(ctx, F);
    M.F = nullptr;
    A->state = M.ldl ? 2 : 1;
    A->k_fail = -1;
    A->eps = M.eps;
    A->flops_exec = M.fl_exec;
    A->flops_model = M.fl_model;
    A->flops_fp32 = M.fl32;
    A->ara_rounds = (double)(M.t32 + M.t64);
    A->tiles_fp32 = M.mixed ? (double)M.t32 : 0.0;
    A->tiles_fp64 = M.mixed ? (double)M.t64 : 0.0;
    A->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - M.t0).count();
    M.done = true;
  }

  void step() {
    step_columns();
    for (auto& Mp : mats) {
      Mat& M = *Mp;
      if (!M.live) {
        if (M.F) {
          free_f32(ctx, M);
          mat_destroy(ctx, M.F);
          M.F = nullptr;
        }
        continue;
      }
      if (M.done || !M.stepped) continue;
      M.stepped = false;
      if (++M.k == M.nb) finalize(M);
    }
    prof_flush(ctx);
  }

  // After the diagonal tiles' join: a tile that is not positive definite fails its matrix, or, with
  // TLR_COMP_MODCHOL, is factored again by Algorithm 8 from its saved copy (main stream).
  void diagonal_failures(int* info) {
    const int nm = (int)mats.size();
    std::vector<int> hinfo(nm);
    TLR_CUDA(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * nm, cudaMemcpyDeviceToHost, ctx->main));
    TLR_CUDA(cudaStreamSynchronize(ctx->main));
    bool redo = false;
    for (int mi = 0; mi < nm; ++mi) {
      Mat& M = *mats[mi];
      if (!M.live || M.done || hinfo[mi] < 0 || M.o.compensation != TLR_COMP_MODCHOL) continue;
      const int b = M.b;
      double* T = static_cast<double*>(M.Asave.p);
      modified_cholesky_tile(ctx, b, T, b, M.F->dinv + (size_t)M.k * b * b, info + mi, bMcW, bMcT);
      copy_matrix(ctx, b, b, T, b, M.F->diag + (size_t)M.k * b * b, b);
      ++M.modified;
      redo = true;
    }
    if (redo) {
      TLR_CUDA(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * nm, cudaMemcpyDeviceToHost, ctx->main));
      TLR_CUDA(cudaStreamSynchronize(ctx->main));
    }
    for (int mi = 0; mi < nm; ++mi) {
      Mat& M = *mats[mi];
      if (M.live && !M.done && hinfo[mi] >= 0) {
        M.live = false;
        M.st = TLR_ERR_NOT_SPD;
        M.A->state = 3;
        M.A->k_fail = M.k;
      }
    }
  }

  // selectPivot (Algorithm 9): for every pivoting matrix not at its last column, the remaining
  // diagonal tile whose updated value A(i,i) - D_i has the largest Frobenius norm (the first on
  // ties); tile rows and columns k and p are exchanged when p != k.
  void select_pivots(const std::vector<Mat*>& L) {
    std::vector<Mat*> P;
    int64_t tot = 0;
    for (Mat* Mp : L)
      if (Mp->piv && Mp->k < Mp->nb - 1) {
        P.push_back(Mp);
        tot += (int64_t)(Mp->nb - Mp->k) * Mp->b;
      }
    if (P.empty()) return;
    double* d = bPiv.need<double>((size_t)tot);
    int64_t o = 0;
    for (Mat* Mp : P) {  // squared norms of the tiles' columns (the tiles are contiguous b x b blocks)
      const int64_t n = (int64_t)(Mp->nb - Mp->k) * Mp->b;
      col_sqnorms(ctx, Mp->F->diag + (size_t)Mp->k * Mp->b * Mp->b, Mp->b, n, d + o);
      o += n;
    }
    std::vector<double> h((size_t)tot);
    TLR_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(double) * tot, cudaMemcpyDeviceToHost, ctx->stream));
    TLR_CUDA(cudaStreamSynchronize(ctx->stream));
    o = 0;
    for (Mat* Mp : P) {
      Mat& M = *Mp;
      int p = M.k;
      double best = -1.0;
      for (int i = M.k; i < M.nb; ++i) {
        double sq = 0.0;
        for (int c = 0; c < M.b; ++c) sq += h[(size_t)o + (size_t)(i - M.k) * M.b + c];
        const double nrm = std::sqrt(sq);
        if (nrm > best) {
          best = nrm;
          p = i;
        }
      }
      o += (int64_t)(M.nb - M.k) * M.b;
      if (p != M.k) exchange_tiles(M, M.k, p);
    }
  }

  // pivotRowColumn (Algorithm 9): exchange tile rows and columns k < p.  The updated diagonal tiles,
  // the points and the permutation swap blocks; F's finished rows k and p (columns j < k) swap their
  // U panels and the positions of their V blocks in each V panel; the compressed input's trailing
  // tiles (i, j), k <= j < i, are rewritten as new(i, j) = old(s(i), s(j)), with s exchanging k and p,
  // or the transpose of old(s(j), s(i)) (U and V exchanged) where the pair crosses the diagonal.  The
  // input's finished columns j < k are no longer read and are released.
  void exchange_tiles(Mat& M, int k, int p) {
    tlr_mat* A = M.A;
    tlr_mat* F = M.F;
    const int nb = M.nb, b = M.b;
    auto sg = [&](int i) { return i == k ? p : (i == p ? k : i); };
    {  // diagonal tiles, ordered points, device permutation: swap block k and block p
      const size_t bb = (size_t)b * b, pb = (size_t)b * A->d;
      double* t = bSwap.need<double>(std::max(bb, pb + (size_t)b));
      auto swap_dev = [&](void* x, void* y, size_t bytes) {
        TLR_CUDA(cudaMemcpyAsync(t, x, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        TLR_CUDA(cudaMemcpyAsync(x, y, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        TLR_CUDA(cudaMemcpyAsync(y, t, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      };
      swap_dev(F->diag + k * bb, F->diag + p * bb, bb * sizeof(double));
      if (A->pts) swap_dev(A->pts + k * pb, A->pts + p * pb, pb * sizeof(double));
      if (A->dperm) swap_dev(A->dperm + (size_t)k * b, A->dperm + (size_t)p * b, (size_t)b * sizeof(int64_t));
      std::swap_ranges(A->perm.begin() + (size_t)k * b, A->perm.begin() + (size_t)(k + 1) * b,
                       A->perm.begin() + (size_t)p * b);
    }
    // ---------------------------------------------------------------- F: rows k and p of columns j < k
    if (k > 0) {
      const std::vector<int> fr = F->rank;
      const std::vector<int64_t> fv = F->voff;
      std::swap(F->Urow[k], F->Urow[p]);
      std::swap(F->ucap[k], F->ucap[p]);
      std::swap(F->ulen[k], F->ulen[p]);
      if (M.oz) {
        std::swap(M.FUs[k], M.FUs[p]);
        std::swap(M.fuscap[k], M.fuscap[p]);
        std::swap(M.FUt[k], M.FUt[p]);
        std::swap(M.futcap[k], M.futcap[p]);
      }
      int64_t seg = 0;
      for (int j = 0; j < k; ++j) {
        std::swap(F->rank[ix(F, k, j)], F->rank[ix(F, p, j)]);
        std::swap(F->uoff[ix(F, k, j)], F->uoff[ix(F, p, j)]);
        seg += F->vlen[j] - fv[ix(F, k, j)];
      }
      // each V panel's rows >= k, staged, then written back block by block in the new row order
      double* t = bSwapV.need<double>((size_t)std::max<int64_t>(seg, 1) * b);
      std::vector<CopyJob> stage, back;
      std::vector<OzColJob> vcj;
      int64_t to = 0;
      for (int j = 0; j < k; ++j) {
        const int64_t s0 = fv[ix(F, k, j)], n = F->vlen[j] - s0;
        if (n <= 0) continue;
        stage.push_back(CopyJob{F->Vcol[j] + (size_t)b * s0, t + (size_t)b * to, n * b});
        int64_t c = s0;
        for (int i = k; i < nb; ++i) {
          const int a = sg(i), r = fr[ix(F, a, j)];
          F->voff[ix(F, i, j)] = c;
          if (r > 0) back.push_back(CopyJob{t + (size_t)b * (to + fv[ix(F, a, j)] - s0), F->Vcol[j] + (size_t)b * c,
                                           (int64_t)r * b});
          c += r;
        }
        to += n;
        if (M.oz && M.FVs[j]) {  // the panel's chunk planes, against its unchanged bound
          OzColJob cj{F->Vcol[j], M.FVs[j], M.dFVe + j, b, (int)F->vlen[j], 0, b};
          cj.emax = M.dFVmax + j;
          vcj.push_back(cj);
        }
      }
      batched_copy(ctx, stage);
      batched_copy(ctx, back);
      oz_split_cols(ctx, vcj);
    }
    // ---------------------------------------------------------------- the compressed input's trailing tiles
    const std::vector<int> ar = A->rank;
    const std::vector<int64_t> au = A->uoff, av = A->voff;
    const std::vector<double*> AU = A->Urow, AV = A->Vcol;
    struct Src {
      const double* U;
      const double* V;
      int r;
    };
    auto src = [&](int i, int j) -> Src {  // the tile at (i, j), i > j >= k, after the exchange
      const int a = sg(i), c = sg(j);
      if (a > c) return Src{AU[a] + (size_t)b * au[ix(A, a, c)], AV[c] + (size_t)b * av[ix(A, a, c)], ar[ix(A, a, c)]};
      return Src{AV[a] + (size_t)b * av[ix(A, c, a)], AU[c] + (size_t)b * au[ix(A, c, a)], ar[ix(A, c, a)]};
    };
    std::vector<CopyJob> cp;
    std::vector<double*> release;
    for (int i = 0; i < nb; ++i) {  // row panels: only the tiles of columns >= k remain
      for (int j = 0; j < std::min(i, k); ++j) {
        A->rank[ix(A, i, j)] = 0;
        A->uoff[ix(A, i, j)] = 0;
        A->voff[ix(A, i, j)] = 0;
      }
      release.push_back(AU[i]);
      A->Urow[i] = nullptr;
      A->ulen[i] = 0;
      A->ucap[i] = 0;
      if (i <= k) continue;
      int64_t len = 0;
      for (int j = k; j < i; ++j) len += src(i, j).r;
      A->Urow[i] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(len, 1) * b));
      A->ulen[i] = len;
      A->ucap[i] = std::max<int64_t>(len, 1);
      int64_t c = 0;
      for (int j = k; j < i; ++j) {
        const Src e = src(i, j);
        A->rank[ix(A, i, j)] = e.r;
        A->uoff[ix(A, i, j)] = c;
        if (e.r > 0) cp.push_back(CopyJob{e.U, A->Urow[i] + (size_t)b * c, (int64_t)e.r * b});
        c += e.r;
      }
    }
    std::vector<OzColJob> acj;
    std::vector<int> acol;
    for (int j = 0; j <= p; ++j) {  // column panels: those of columns k..p change, those before k go
      if (j >= k && j == nb - 1) continue;
      release.push_back(AV[j]);
      A->Vcol[j] = nullptr;
      A->vlen[j] = 0;
      if (M.oz) {
        dfree(ctx, M.AVs[j]);
        M.AVs[j] = nullptr;
      }
      if (j < k) continue;
      int64_t len = 0;
      for (int i = j + 1; i < nb; ++i) len += src(i, j).r;
      A->Vcol[j] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(len, 1) * b));
      A->vlen[j] = len;
      int64_t c = 0;
      for (int i = j + 1; i < nb; ++i) {
        const Src e = src(i, j);
        A->voff[ix(A, i, j)] = c;
        if (e.r > 0) cp.push_back(CopyJob{e.V, A->Vcol[j] + (size_t)b * c, (int64_t)e.r * b});
        c += e.r;
      }
      if (M.oz && len > 0) {
        M.AVs[j] = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * len));
        OzColJob cj{A->Vcol[j], M.AVs[j], M.dAVe + j, b, (int)len, 0, b};
        cj.emax = M.dAVmax + j;
        acj.push_back(cj);
        acol.push_back(j);
      }
    }
    batched_copy(ctx, cp);
    for (double* q : release) dfree(ctx, q);
    for (int j : acol) oz_absmax(ctx, 1, (int64_t)b * A->vlen[j], A->Vcol[j], M.dAVmax + j);
    oz_split_cols(ctx, acj);
  }

  // denseUpdates (Algorithm 9): once column k is final, every later diagonal tile of a pivoting matrix
  // takes its term, A(i,i) -= U_ik (V_ikᵀ V_ik) U_ikᵀ, so that at the next step the tiles hold
  // A(i,i) - D_i for the pivot selection (whole tiles: the norm is that of the symmetric tile).  The
  // Gram factor and E = U_ik G are FP64 GEMMs.  The b x b update A(i,i) -= E U_ik^T is an FP64 GEMM
  // for ranks below 32 and a product on the tensor cores by exact splitting otherwise (tiles of a
  // multiple of 16): with K = r that small, the split product's per-block cost (a 128 x 16 FP64 output
  // block read and written per CTA) exceeds the 2 b^2 r FP64 flops (C3 at eps 1e-2: 1.01 s against
  // 1.21 s all split; C2 at eps 1e-8, ranks ~100: 1.54 s all FP64 against 1.49 s).  For the split
  // products E = -U_ik G is split per tile against its own bound (a matrix's blocks padded to its
  // largest split rank of the step, so that one launch takes every bound) and U_ik, whose columns are
  // orthonormal, transposed against the fixed bound 2.
  void pivot_dense_updates(const std::vector<Mat*>& L) {
    struct Up {
      Mat* M;
      int i, r;
      int64_t go, eo;
      bool sp;  // the update on the tensor cores
    };
    auto split = [](const Mat& M, int r) { return M.oz && r >= 32; };
    std::vector<Up> ups;
    std::vector<int64_t> rmax(L.size(), 0), ebase(L.size(), 0);
    int64_t gt = 0, et = 0, nsp = 0;
    for (size_t u = 0; u < L.size(); ++u) {
      Mat& M = *L[u];
      if (!M.piv || !M.live || M.nops == 0) continue;
      for (int i = M.k + 1; i < M.nb; ++i) {
        const int r = M.F->rank[ix(M.F, i, M.k)];
        if (split(M, r)) rmax[u] = std::max<int64_t>(rmax[u], r);
      }
      ebase[u] = et;
      for (int i = M.k + 1; i < M.nb; ++i) {  // the split blocks first: contiguous for their bounds
        const int r = M.F->rank[ix(M.F, i, M.k)];
        if (r == 0 || !split(M, r)) continue;
        ups.push_back(Up{&M, i, r, gt, et, true});
        gt += (int64_t)r * r;
        et += (int64_t)M.b * rmax[u];
        ++nsp;
      }
      for (int i = M.k + 1; i < M.nb; ++i) {
        const int r = M.F->rank[ix(M.F, i, M.k)];
        if (r == 0 || split(M, r)) continue;
        ups.push_back(Up{&M, i, r, gt, et, false});
        gt += (int64_t)r * r;
        et += (int64_t)M.b * r;
      }
    }
    if (ups.empty()) return;
    double* G = bPivG.need<double>((size_t)gt);
    double* E = bPivE.need<double>((size_t)et);
    if (nsp) TLR_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * (size_t)et, ctx->stream));  // zero padding
    std::vector<GemmJob<double>> jg, je, jd;
    for (const Up& w : ups) {
      Mat& M = *w.M;
      tlr_mat* F = M.F;
      const int b = M.b, r = w.r;
      const double* U = Uptr(F, w.i, M.k);
      const double* V = Vptr(F, w.i, M.k);
      jg.push_back(job<double>(TN, r, r, V, b, V, b, b, G + w.go, r, 1.0, 0.0));
      je.push_back(job<double>(NN, b, r, U, b, G + w.go, r, r, E + w.eo, b, w.sp ? -1.0 : 1.0, 0.0));
      if (!w.sp)
        jd.push_back(job<double>(NT, b, b, E + w.eo, b, U, b, r, F->diag + (size_t)w.i * b * b, b, -1.0, 1.0));
      M.fl_exec += 2.0 * b * r * r * 2.0 + 2.0 * b * b * r;
    }
    gemm<double>(ctx, TN, jg);
    gemm<double>(ctx, NN, je);
    gemm<double>(ctx, NT, jd);
    if (nsp == 0) return;
    // chunk planes: E (columns along b, acol) and U_ik^T (rows along its r columns, padded to 16)
    int64_t pe = 0, pu = 0;
    for (const Up& w : ups)
      if (w.sp) {
        pe += (int64_t)8 * w.M->b * w.r;
        pu += (int64_t)8 * w.M->b * oz_ld(w.r);
      }
    int8_t* Es = bPivS.need<int8_t>((size_t)(pe + pu));
    int8_t* Us = Es + pe;
    unsigned long long* em = bPivX.need<unsigned long long>((size_t)nsp * 2);
    int* ee = reinterpret_cast<int*>(em + nsp);
    TLR_CUDA(cudaMemsetAsync(Us, 0, (size_t)pu, ctx->stream));
    std::vector<OzColJob> cj;
    std::vector<OzJob> dj;
    int64_t oe = 0, ou = 0, t = 0;
    for (size_t u = 0; u < L.size(); ++u) {  // one bound per E block, one launch per matrix
      Mat& M = *L[u];
      if (!M.piv || !M.live || M.nops == 0 || !M.oz) continue;
      int64_t nblk = 0;
      for (const Up& w : ups) nblk += (w.M == &M && w.sp) ? 1 : 0;
      if (nblk) oz_absmax(ctx, (int)nblk, (int64_t)M.b * rmax[u], E + ebase[u], em + t);
      t += nblk;
    }
    t = 0;
    for (const Up& w : ups) {
      Mat& M = *w.M;
      if (!w.sp) continue;
      const int b = M.b, r = w.r, tl = oz_ld(r);
      OzColJob ce{E + w.eo, Es + oe, ee + t, b, r, 0, b};
      ce.emax = em + t;
      cj.push_back(ce);
      OzColJob cu{Uptr(M.F, w.i, M.k), Us + ou, nullptr, b, r, 0, b};
      cu.plane = (size_t)b * tl;
      cu.efix = 1;
      cu.tld = tl;
      cj.push_back(cu);
      OzJob d{Es + oe, Us + ou, ee + t, d_one, M.F->diag + (size_t)w.i * b * b, (size_t)b * r, (size_t)b * tl, b, b, b,
              b, r};
      d.acol = 1;
      d.ldb = tl;
      d.eB_stride = 0;
      d.accumulate = 1;
      dj.push_back(d);
      oe += (int64_t)8 * b * r;
      ou += (int64_t)8 * b * tl;
      ++t;
    }
    oz_split_cols(ctx, cj);
    oz_gemm(ctx, dj);
  }

  void step_columns() {
    std::vector<Mat*> L;
    for (auto& M : mats)
      if (M->live && !M->done) L.push_back(M.get());
    if (L.empty()) return;
    select_pivots(L);
    // ---------------------------------------------------------------- Gram factors
    prof_mark(ctx, PH_GRAM);
    {
      std::vector<GemmJob<double>> jg;
      std::vector<GemmJob<float>> jg32;
      std::vector<ScaleJob> sj;
      std::vector<ConvJob> cdv;
      std::vector<OzJob> ogj;      // split Gram products
      std::vector<OzColJob> dvcj;  // LDL^T: slices of D_j V_kj
      int8_t* dvs_ = nullptr;
      int* dve_ = nullptr;
      {
        int64_t el = 0, ex = 0;
        for (Mat* Mp : L)
          if (Mp->ldl && Mp->oz)
            for (int j = 0; j < Mp->k; ++j) {
              const int r = Mp->F->rank[ix(Mp->F, Mp->k, j)];
              el += (int64_t)8 * Mp->b * r;
              ex += r;
            }
        if (el) {
          dvs_ = bOzOs.need<int8_t>((size_t)el);
          dve_ = bOzOe.need<int>((size_t)ex);
        }
      }
      for (Mat* Mp : L) {
        Mat& M = *Mp;
        tlr_mat* F = M.F;
        const int b = M.b;
        M.Kk = (int)F->ulen[M.k];
        M.R0k = M.A->vlen[M.k];
        M.goff.assign(std::max(M.k, 1), 0);
        M.gld.assign(std::max(M.k, 1), 1);
        M.gtot = 0;
        int64_t dvtot = 0;
        for (int j = 0; j < M.k; ++j) {
          M.goff[j] = M.gtot;
          M.gld[j] = (int)std::max<int64_t>(1, F->vlen[j] - F->voff[ix(F, M.k, j)]);
          M.gtot += (int64_t)M.gld[j] * F->rank[ix(F, M.k, j)];
          dvtot += (int64_t)b * F->rank[ix(F, M.k, j)];
        }
        double* G = M.G.need<double>((size_t)std::max<int64_t>(M.gtot, 1));
        float* G32 = M.mixed ? M.G32.need<float>((size_t)std::max<int64_t>(M.gtot, 1)) : nullptr;
        double* DV = M.ldl ? M.DV.need<double>((size_t)std::max<int64_t>(dvtot, 1)) : nullptr;
        float* DV32 = (M.ldl && M.mixed) ? M.DV32.need<float>((size_t)std::max<int64_t>(dvtot, 1)) : nullptr;
        int64_t dvo = 0;
        for (int j = 0; j < M.k; ++j) {
          const int rkj = F->rank[ix(F, M.k, j)];
          if (rkj == 0) continue;
          const int S = (int)(F->vlen[j] - F->voff[ix(F, M.k, j)]);
          const double* Vkj = Vptr(F, M.k, j);
          const float* Vkj32 = M.mixed ? M.FV32[j] + (size_t)b * F->voff[ix(F, M.k, j)] : nullptr;
          if (M.ldl) {  // D_j V_kj (Equation 3: D(j,j) inside the chain)
            sj.push_back(ScaleJob{F->dvec + (size_t)j * b, Vkj, DV + dvo, b, rkj, b, b, 0});
            Vkj = DV + dvo;
            if (M.mixed) {
              cdv.push_back(ConvJob{DV + dvo, DV32 + dvo, (int64_t)b * rkj});
              Vkj32 = DV32 + dvo;
            }
            dvo += (int64_t)b * rkj;
          }
          if (M.oz && M.FVs[j]) {  // G = Vcol_j[i >= k]^T [D_j] V_kj on the tensor cores
            const size_t vo = (size_t)b * F->voff[ix(F, M.k, j)], pl = (size_t)b * F->vlen[j];
            OzJob gj{M.FVs[j] + vo, M.FVs[j] + vo, M.dFVe + j, M.dFVe + j, G + M.goff[j], pl, pl, b, M.gld[j],
                     S, rkj, b};
            gj.ldb = b;
            gj.eB_stride = 0;
            if (M.ldl) {  // B = D_j V_kj: its own slices, per column
              gj.B = dvs_ + 0;
              gj.sB = (size_t)b * rkj;
              gj.eB = dve_;
              gj.eB_stride = 1;
              dvcj.push_back(OzColJob{Vkj, dvs_, dve_, b, rkj, 0, b});
              dvs_ += (size_t)8 * b * rkj;
              dve_ += rkj;
            }
            ogj.push_back(gj);
          } else {
            jg.push_back(job<double>(TN, S, rkj, Vptr(F, M.k, j), b, Vkj, b, b, G + M.goff[j], M.gld[j], 1.0, 0.0));
          }
          M.fl_exec += 2.0 * b * S * rkj;
          if (M.mixed)  // FP32 Gram for the tiles that sample in FP32
            jg32.push_back(job<float>(TN, S, rkj, M.FV32[j] + (size_t)b * F->voff[ix(F, M.k, j)], b, Vkj32, b, b,
                                      G32 + M.goff[j], M.gld[j], 1.0, 0.0));
        }
      }
      batched_scale_rows(ctx, sj);
      batched_to_float(ctx, cdv);
      gemm<double>(ctx, TN, jg);
      gemm<float>(ctx, TN, jg32);
      oz_split_cols(ctx, dvcj);
      oz_gemm(ctx, ogj);
    }
    // ---------------------------------------------------------------- diagonal tiles (side stream)
    // The diagonal tile is read by the column's batchTrsm only, not by its ARA: its
    // updateDense, chol / LDL^T and inverse run on the side stream, overlapped with the
    // sampling rounds, and join before the trsm.  (Schur compensation runs a nested ARA
    // with its own workspaces and stays on the main stream.)
    const int nm = (int)mats.size();
    int* info = bInfo.need<int>((size_t)nm);
    // updateDense on the tensor cores (side stream): D_k += E Urow_k^T with E = -[U_kj G_kj]_j split into
    // chunk planes per column and the transposed U-panel planes as the right operand; exact integer totals
    // need K <= 16384
    auto dense_split = [&](const Mat& M) {
      return M.o.compensation != TLR_COMP_SCHUR && M.oz && !M.piv && M.Kk > 0 && M.Kk <= 16384;
    };
    int8_t* dsp = nullptr;
    int* dse = nullptr;
    unsigned long long* dsm = nullptr;
    {  // the side stream must not reallocate its workspace: size it here
      std::vector<DenseTile> probe[2];
      int64_t del = 0, dn = 0;
      for (Mat* Mp : L) {
        if (Mp->o.compensation != TLR_COMP_SCHUR)
          probe[Mp->ldl].push_back(DenseTile{nullptr, nullptr, nullptr, Mp->F->dinv, Mp->b, Mp->b});
        if (dense_split(*Mp)) {
          del += (int64_t)8 * Mp->b * Mp->Kk;
          ++dn;
        }
        if (Mp->o.compensation == TLR_COMP_MODCHOL) Mp->Asave.need<double>((size_t)Mp->b * Mp->b);
      }
      bTmp.need<double>(std::max(dense_tmp_doubles(probe[0], 0), dense_tmp_doubles(probe[1], 1)));
      if (dn) {
        dsp = bOzDs.need<int8_t>((size_t)del);
        dse = bOzDe.need<int>((size_t)dn);
        dsm = bOzDm.need<unsigned long long>((size_t)dn);
      }
    }
    TLR_CUDA(cudaMemsetAsync(info, 0xff, sizeof(int) * nm, ctx->main));
    TLR_CUDA(cudaEventRecord(ctx->ev_fork, ctx->main));
    TLR_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    for (int pass = 0; pass < 2; ++pass) {
      // pass 0: matrices without Schur compensation, on the side stream; pass 1: the others, main stream
      std::vector<Mat*> S;
      for (Mat* Mp : L)
        if ((Mp->o.compensation == TLR_COMP_SCHUR) == (pass == 1)) S.push_back(Mp);
      if (S.empty()) continue;
      ctx->stream = pass == 0 ? ctx->side : ctx->main;
      std::vector<GemmJob<double>> je, jd;
      std::vector<OzColJob> ecj;  // split updateDense: slices of E
      std::vector<OzJob> edj;
      std::vector<std::pair<const double*, int64_t>> emx;  // E blocks whose bound is taken
      std::vector<DiagJob> shifts;
      std::vector<DenseTile> tiles[2];  // by factorization kind (Cholesky, LDL^T)
      for (Mat* Mp : S) {
        Mat& M = *Mp;
        tlr_mat* F = M.F;
        const int b = M.b;
        double* Akk = F->diag + (size_t)M.k * b * b;
        const double* G = static_cast<const double*>(M.G.p);
        if (M.Kk > 0 && !M.piv) {  // with tile pivoting D_k is already in the tile
          double* E = M.E.need<double>((size_t)b * M.Kk);
          const bool sp = pass == 0 && dense_split(M);
          for (int j = 0; j < M.k; ++j) {
            const int rkj = F->rank[ix(F, M.k, j)];
            if (rkj == 0) continue;
            je.push_back(job<double>(NN, b, rkj, Uptr(F, M.k, j), b, G + M.goff[j], M.gld[j], rkj,
                                     E + (size_t)b * F->uoff[ix(F, M.k, j)], b, sp ? -1.0 : 1.0, 0.0));
            M.fl_exec += 2.0 * b * rkj * rkj;
          }
          if (sp) {  // D_k += E Urow_k^T, E(m, k) read along m (its own column-major layout)
            emx.push_back({E, (int64_t)b * M.Kk});
            OzColJob c{E, dsp, dse, b, (int)M.Kk, 0, b};
            c.emax = dsm;
            ecj.push_back(c);
            OzJob d{dsp, M.FUt[M.k], dse, d_one, Akk, (size_t)b * M.Kk, (size_t)b * M.futcap[M.k], b, b, b, b,
                    (int)M.Kk};
            d.acol = 1;
            d.ldb = (int)M.futcap[M.k];
            d.eB_stride = 0;
            d.accumulate = 1;
            edj.push_back(d);
            dsp += (size_t)8 * b * M.Kk;
            ++dse;
            ++dsm;
            M.fl_exec += 2.0 * b * b * M.Kk;  // the whole tile (the factorization reads its lower triangle)
          } else {
            GemmJob<double> g = job<double>(NT, b, b, E, b, F->Urow[M.k], b, M.Kk, Akk, b, -1.0, 1.0);
            if (pass == 0) g.flags = GEMM_TRIL;
            M.fl_exec += (pass == 0 ? 1.0 : 2.0) * b * b * M.Kk;
            if (pass == 1) {  // full D_k into a scratch tile for the compensation
              g.C = static_cast<double*>(M.DV.need<double>((size_t)b * b));  // reuse: D_k
              g.alpha = 1.0;
              g.beta = 0.0;
            }
            jd.push_back(g);
          }
        }
        if (M.o.compensation == TLR_COMP_SHIFT && M.o.shift != 0.0 && !M.piv)
          shifts.push_back(DiagJob{Akk, b, b, M.o.shift});
        int mi = 0;
        for (; mi < nm; ++mi)
          if (mats[mi].get() == Mp) break;
        tiles[M.ldl].push_back(DenseTile{Akk, M.ldl ? F->dvec + (size_t)M.k * b : nullptr, info + mi,
                                  F->dinv + (size_t)M.k * b * b, b, b});
        M.fl_exec += 2.0 * (double)b * b * b / 3.0;
        M.fl_model += (double)b * b * b / 3.0;
        for (int j = 0; j < M.k; ++j) {
          const int r = F->rank[ix(F, M.k, j)];
          M.fl_model += 4.0 * b * r * r + 2.0 * b * b * r;
        }
      }
      gemm<double>(ctx, NN, je);
      gemm<double>(ctx, NT, jd);
      if (!edj.empty()) {
        unsigned long long* m0 = static_cast<unsigned long long*>(bOzDm.p);
        for (size_t u = 0; u < emx.size(); ++u) oz_absmax(ctx, 1, emx[u].second, emx[u].first, m0 + u);
        oz_split_cols(ctx, ecj);
        oz_gemm(ctx, edj);
      }
      if (pass == 1) {
        // Section 5.1.1: A_kk - D_k + diag(rowsum |D_k - Dbar_k|), Dbar_k = Q Q^T D_k Q Q^T,
        // Q the eps-basis of D_k from ARA.
        for (Mat* Mp : S) {
          Mat& M = *Mp;
          if (M.Kk == 0) continue;
          const int b = M.b;
          double* Akk = M.F->diag + (size_t)M.k * b * b;
          double* Dk = static_cast<double*>(M.DV.p);
          axpy_matrix(ctx, b, b, -1.0, Dk, b, Akk, b);
          Buf bq(ctx), bb(ctx), bc(ctx);
          double* Qd = bq.need<double>((size_t)b * (b + bs));
          double* Bd = bb.need<double>((size_t)b * b);
          double* C1 = bc.need<double>((size_t)2 * b * b);
          double* C2 = C1 + (size_t)b * b;
          std::vector<int> qd;
          AraStats as;
          ara_dense_run(ctx, 1, b, Dk, bs, M.eps, M.o.seed, STREAM_SCHUR, (uint32_t)M.k, Qd, Bd, qd, as);
          const int r = qd[0];
          if (r > 0) {  // Bd = D Q (D symmetric): C1 = Q^T Bd, C2 = Q C1, E = D - C2 Q^T
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
      batched_add_diag(ctx, shifts);
      for (Mat* Mp : S)  // Algorithm 8 needs the tile as it was before the factorization attempt
        if (Mp->o.compensation == TLR_COMP_MODCHOL)
          copy_matrix(ctx, Mp->b, Mp->b, Mp->F->diag + (size_t)Mp->k * Mp->b * Mp->b, Mp->b,
                      static_cast<double*>(Mp->Asave.p), Mp->b);
      // pass 1 runs on the main stream while pass 0 may still be running: own workspace
      Buf& tmp = pass == 0 ? bTmp : bTmpMain;
      for (int l = 0; l < 2; ++l) {
        dense_factor_batch(ctx, tiles[l], l, tmp);
        dense_trinv_batch(ctx, tiles[l], l, tmp);
      }
    }
    TLR_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
    ctx->stream = ctx->main;
    // ---------------------------------------------------------------- cholARAUpdate (Algorithm 5)
    std::vector<int> op_m, op_i, nrow, order;
    std::vector<double> thr;
    std::vector<int64_t> qoff;
    int64_t qtot = 0;
    for (size_t u = 0; u < L.size(); ++u) {
      Mat& M = *L[u];
      M.op0 = (int)op_m.size();
      M.nops = M.nb - M.k - 1;
      std::vector<int> ord(M.nops);
      std::iota(ord.begin(), ord.end(), 0);
      // tiles enter the batch by their original rank, descending (Algorithm 5 sortRanks)
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) {
        return M.A->rank[ix(M.A, M.k + 1 + a, M.k)] > M.A->rank[ix(M.A, M.k + 1 + c, M.k)];
      });
      for (int v : ord) order.push_back(M.op0 + v);
      for (int v = 0; v < M.nops; ++v) {
        op_m.push_back((int)u);
        op_i.push_back(M.k + 1 + v);
        nrow.push_back(M.b);
        thr.push_back(M.thr);
        qoff.push_back(qtot);
        qtot += (int64_t)M.b * (M.b + bs);
      }
    }
    const int nops = (int)op_m.size();
    std::vector<int> q(nops, 0);
    double* Q = bQ.need<double>((size_t)std::max<int64_t>(qtot, 1));
    if (nops > 0) {
      // device tables of every matrix (ranks and offsets of F, Gram offsets of this column)
      // Each matrix's region: rank/uoff/voff (3 nb^2 ints), then the int64 Gram offsets at
      // an even int offset (8-byte aligned), then the Gram leading dimensions; every
      // region starts at an even offset as well.
      auto even = [](int64_t v) { return (v + 1) & ~int64_t(1); };
      std::vector<int64_t> toff(L.size()), g0(L.size());
      int64_t tint = 0;
      for (size_t u = 0; u < L.size(); ++u) {
        const int64_t kk = std::max(L[u]->k, 1);
        toff[u] = tint;
        g0[u] = even((int64_t)3 * L[u]->nb * L[u]->nb);
        tint += even(g0[u] + 3 * kk);
      }
      std::vector<int> htab((size_t)tint, 0);
      for (size_t u = 0; u < L.size(); ++u) {
        Mat& M = *L[u];
        tlr_mat* F = M.F;
        const int nb2 = M.nb * M.nb;
        const int kk = std::max(M.k, 1);
        int* t = htab.data() + toff[u];
        for (int e = 0; e < nb2; ++e) {
          t[e] = F->rank[e];
          t[nb2 + e] = (int)F->uoff[e];
          t[2 * nb2 + e] = (int)F->voff[e];
        }
        int64_t* go = reinterpret_cast<int64_t*>(t + g0[u]);
        for (int j = 0; j < kk; ++j) go[j] = M.goff[j];
        int* gl = t + g0[u] + 2 * kk;
        for (int j = 0; j < kk; ++j) gl[j] = M.gld[j];
      }
      int* dtab = bTab.need<int>((size_t)tint + 2);
      TLR_CUDA(cudaMemcpyAsync(dtab, htab.data(), sizeof(int) * tint, cudaMemcpyHostToDevice, ctx->stream));
      TLR_CUDA(cudaStreamSynchronize(ctx->stream));  // htab is pageable
      for (size_t u = 0; u < L.size(); ++u) {
        Mat& M = *L[u];
        const int kk = std::max(M.k, 1);
        M.dtab = dtab + toff[u];
        M.dgoff = reinterpret_cast<const int64_t*>(dtab + toff[u] + g0[u]);
        M.dgld = dtab + toff[u] + g0[u] + 2 * kk;
      }
      // per-tile precision rule (mixed precision): FP32 when u32 sqrt(K)(|A_ik|_F + sum_j
      // |L_ij|_F |L_kj|_F) <= thr / 8, else FP64
      std::vector<char> is32(nops, 0), is64(nops, 1);
      bool any32 = false;
      for (int op = 0; op < nops; ++op) {
        Mat& M = *L[op_m[op]];
        if (!M.mixed) continue;
        const int i = op_i[op];
        double sum = M.nA[ix(M.A, i, M.k)];
        for (int j = 0; j < M.k; ++j) sum += M.nL[ix(M.F, i, j)] * M.nL[ix(M.F, M.k, j)];
        const double K = (double)M.A->rank[ix(M.A, i, M.k)] + (double)M.F->ulen[i] + bs;
        if (U32 * std::sqrt(K) * sum <= M.thr / 8.0) {
          is32[op] = 1;
          is64[op] = 0;
          any32 = true;
        }
      }
      BatchSampler<double> s64;
      BatchSampler<float> s32;
      auto setup = [&](auto& S, const std::vector<char>* mem) {
        S.ctx = ctx; S.bs = bs; S.L = &L; S.op_m = &op_m; S.op_i = &op_i; S.member = mem;
        S.Q = Q; S.qoff = &qoff;
        S.bom = &bOm; S.bom32 = &bOm32; S.bw = &bW; S.by32 = &bY32; S.bp = &bP; S.bz = &bZ;
        S.bq32 = &bQ32; S.bb32 = &bB32;
        S.d_one = d_one; S.bos = &bOzOs; S.boe = &bOzOe; S.bws = &bOzWs; S.bwe = &bOzWe; S.bu0 = &bOzU0;
        S.bu0p = &bOzU0p;
      };
      setup(s64, any32 ? &is64 : nullptr);
      setup(s32, &is32);
      SplitSampler split;
      split.f64 = &s64;
      split.f32 = &s32;
      split.is32 = &is32;
      Sampler* smp = any32 ? static_cast<Sampler*>(&split) : static_cast<Sampler*>(&s64);
      // the projection runs after the join (Bc is allocated once the ranks are known)
      struct Deferred : Sampler {
        Sampler* f;
        bool owns_omega() const override { return true; }
        void sample(const std::vector<int>& ops, int t, const double* Om, const std::vector<double*>& Y) override {
          f->sample(ops, t, Om, Y);
        }
        void project(const std::vector<int>&) override {}
      } dsmp;
      dsmp.f = smp;
      int max_slots = 0;
      for (Mat* Mp : L) max_slots += Mp->o.max_slots > 0 ? Mp->o.max_slots : Mp->nb;
      AraConfig cf{bs, 0, STREAM_FACTOR, 0, max_slots};
      cf.fused_all = true;  // slot results independent of the batch
      AraStats as;
      ara_run(ctx, dsmp, nrow, thr, cf, order, Q, qoff, q, as);
      total.rounds += as.rounds;
      total.flops += as.flops;
      // orthogonalization flops, attributed per matrix by its share of the operands
      for (size_t u = 0; u < L.size(); ++u)
        if (nops) L[u]->fl_exec += as.flops * (double)L[u]->nops / nops;
      // ---------------------------------------------------------------- join, failures
      prof_mark(ctx, PH_POTRF);  // waiting for the diagonal tiles
      TLR_CUDA(cudaStreamWaitEvent(ctx->main, ctx->ev_join, 0));
      diagonal_failures(info);
      // ---------------------------------------------------------------- projection (sampleLeftT)
      prof_mark(ctx, PH_PROJECT);
      for (Mat* Mp : L) {
        Mat& M = *Mp;
        M.boff.assign(M.nops, 0);
        M.Rk = 0;
        for (int v = 0; v < M.nops; ++v) {
          M.boff[v] = M.Rk;
          M.Rk += M.live ? q[M.op0 + v] : 0;
        }
        M.Bc.need<double>((size_t)std::max<int64_t>(M.Rk, 1) * M.b);
      }
      // failed matrices are not projected
      std::vector<char> keep(nops, 1);
      for (int op = 0; op < nops; ++op) keep[op] = L[op_m[op]]->live;
      std::vector<char> k64(nops), k32(nops);
      for (int op = 0; op < nops; ++op) {
        k64[op] = keep[op] && is64[op];
        k32[op] = keep[op] && is32[op];
      }
      s64.member = &k64;
      s32.member = &k32;
      s64.project(q);
      if (any32) s32.project(q);
    } else {
      prof_mark(ctx, PH_POTRF);
      TLR_CUDA(cudaStreamWaitEvent(ctx->main, ctx->ev_join, 0));
      diagonal_failures(info);
    }
    // ---------------------------------------------------------------- batchTrsm, updateTiles
    prof_mark(ctx, PH_TRSM);
    std::vector<GemmJob<double>> jt;
    std::vector<ScaleJob> sj;
    // V_ik = L_kk^{-1} B_i (LDL^T: then D_k^{-1}, batchIDMult).  L_kk^{-1} is a dense tile and
    // B the column's stacked projections: for tiles of a multiple of 8 the product runs on the
    // tensor cores by exact splitting (k_ozaki.cu), like the construction's products.
    std::vector<Mat*> split;
    int64_t scols = 0;
    for (Mat* Mp : L) {
      Mat& M = *Mp;
      if (!M.live || M.nops == 0) continue;
      tlr_mat* F = M.F;
      const int b = M.b;
      F->Vcol[M.k] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(M.Rk, 1) * b));
      F->vlen[M.k] = M.Rk;
      if (M.Rk > 0) {
        if (b % 16 == 0) {
          split.push_back(Mp);
          scols += M.Rk;
        } else {
          GemmJob<double> g = job<double>(NN, b, (int)M.Rk, F->dinv + (size_t)M.k * b * b, b,
                                          static_cast<double*>(M.Bc.p), b, b, F->Vcol[M.k], b, 1.0, 0.0);
          g.flags = GEMM_ALOWER;  // L_kk^{-1} is lower triangular
          jt.push_back(g);
        }
        if (M.ldl) sj.push_back(ScaleJob{F->dvec + (size_t)M.k * b, F->Vcol[M.k], F->Vcol[M.k], b, (int)M.Rk, b, b, 1});
        M.fl_exec += (double)b * (b + 1) * M.Rk;
        M.fl_model += (double)b * b * M.Rk;
      }
    }
    gemm<double>(ctx, NN, jt);
    if (!split.empty()) {
      const int ns = (int)split.size();
      int64_t tel = 0;
      for (Mat* Mp : split) tel += (int64_t)Mp->b * Mp->b;
      unsigned long long* tmax = bOzMax.need<unsigned long long>((size_t)ns);
      int8_t* Sr = bOzS.need<int8_t>((size_t)8 * tel);
      int* eT = bOzE.need<int>((size_t)ns);
      int64_t xel = 0;
      for (Mat* Mp : split) xel += (int64_t)8 * Mp->b * Mp->Rk;
      int8_t* Xs = bOzX.need<int8_t>((size_t)std::max<int64_t>(xel, 1));
      int* ex = bOzEx.need<int>((size_t)scols);
      std::vector<OzColJob> cj;
      std::vector<OzJob> oj;
      int64_t to = 0, co = 0, xo = 0;
      for (int u = 0; u < ns; ++u) {
        Mat& M = *split[u];
        const int b = M.b;
        const double* Li = M.F->dinv + (size_t)M.k * b * b;
        oz_absmax(ctx, 1, (int64_t)b * b, Li, tmax + u);
        oz_split_tiles(ctx, 1, b, Li, tmax + u, nullptr, Sr + 8 * to, eT + u);
        cj.push_back(OzColJob{static_cast<double*>(M.Bc.p), Xs + xo, ex + co, b, (int)M.Rk, 0, b});
        oj.push_back(OzJob{Sr + 8 * to, Xs + xo, eT + u, ex + co, M.F->Vcol[M.k], (size_t)b * b,
                           (size_t)b * M.Rk, b, b, b, (int)M.Rk, b});
        to += (int64_t)b * b;
        co += M.Rk;
        xo += (int64_t)8 * b * M.Rk;
      }
      oz_split_cols(ctx, cj);
      oz_gemm(ctx, oj);
    }
    batched_scale_rows(ctx, sj);
    {  // slices of the new V panels for the Gram products of the later columns
      std::vector<OzColJob> vcj;
      for (Mat* Mp : L) {
        Mat& M = *Mp;
        if (!M.live || M.nops == 0 || !M.oz || M.Rk == 0) continue;
        const int b = M.b;
        M.FVs[M.k] = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * M.Rk));
        oz_absmax(ctx, 1, (int64_t)b * M.Rk, M.F->Vcol[M.k], M.dFVmax + M.k);
        OzColJob c{M.F->Vcol[M.k], M.FVs[M.k], M.dFVe + M.k, b, (int)M.Rk, 0, b};
        c.emax = M.dFVmax + M.k;
        vcj.push_back(c);
      }
      oz_split_cols(ctx, vcj);
    }
    prof_mark(ctx, PH_UPDATE);
    std::vector<CopyJob> cj;
    std::vector<ConvJob> c32;
    std::vector<OzColJob> usl;  // slices of the appended U blocks
    for (Mat* Mp : L) {
      Mat& M = *Mp;
      if (!M.live || M.nops == 0) continue;
      tlr_mat* F = M.F;
      const int b = M.b;
      for (int v = 0; v < M.nops; ++v) {
        const int op = M.op0 + v, i = M.k + 1 + v, r = q[op];
        ensure_ucap(ctx, F, i, r);
        F->rank[ix(F, i, M.k)] = r;
        F->uoff[ix(F, i, M.k)] = F->ulen[i];
        F->voff[ix(F, i, M.k)] = M.boff[v];
        cj.push_back(CopyJob{Q + qoff[op], F->Urow[i] + (size_t)F->ulen[i] * b, (int64_t)r * b});
        if (M.mixed) {
          if (F->ulen[i] + r > M.fu32cap[i]) {  // grow the FP32 copy of block row i
            const int64_t cap = std::max<int64_t>(F->ucap[i], F->ulen[i] + r);
            float* p = f32_alloc(ctx, (int64_t)b * cap);
            if (F->ulen[i] > 0)
              TLR_CUDA(cudaMemcpyAsync(p, M.FU32[i], sizeof(float) * (size_t)b * F->ulen[i],
                                       cudaMemcpyDeviceToDevice, ctx->stream));
            dfree(ctx, M.FU32[i]);
            M.FU32[i] = p;
            M.fu32cap[i] = cap;
          }
          c32.push_back(ConvJob{Q + qoff[op], M.FU32[i] + (size_t)F->ulen[i] * b, (int64_t)r * b});
        }
        if (M.oz && r > 0) {
          if (F->ulen[i] + r > M.fuscap[i]) {  // grow the slices of block row i (8 planes)
            const int64_t cap = std::max<int64_t>(F->ucap[i], F->ulen[i] + r);
            int8_t* p = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * cap));
            if (F->ulen[i] > 0)
              TLR_CUDA(cudaMemcpy2DAsync(p, (size_t)b * cap, M.FUs[i], (size_t)b * M.fuscap[i],
                                         (size_t)b * F->ulen[i], 8, cudaMemcpyDeviceToDevice,
                                         ctx->stream));
            dfree(ctx, M.FUs[i]);
            M.FUs[i] = p;
            M.fuscap[i] = cap;
          }
          OzColJob sjb{Q + qoff[op], M.FUs[i] + (size_t)F->ulen[i] * b, nullptr, b, r, 0, b};
          sjb.plane = (size_t)b * M.fuscap[i];
          sjb.efix = 1;
          usl.push_back(sjb);
          if (F->ulen[i] + r > M.futcap[i]) {  // grow the transposed planes (rows keep their columns)
            const int64_t cap = oz_ld((int)std::max<int64_t>(F->ucap[i], F->ulen[i] + r));
            int8_t* p = static_cast<int8_t*>(dalloc(ctx, 8 * (size_t)b * cap));
            TLR_CUDA(cudaMemsetAsync(p, 0, 8 * (size_t)b * cap, ctx->stream));
            if (F->ulen[i] > 0)
              TLR_CUDA(cudaMemcpy2DAsync(p, (size_t)cap, M.FUt[i], (size_t)M.futcap[i], (size_t)F->ulen[i],
                                         (size_t)8 * b, cudaMemcpyDeviceToDevice, ctx->stream));
            dfree(ctx, M.FUt[i]);
            M.FUt[i] = p;
            M.futcap[i] = cap;
          }
          OzColJob tjb{Q + qoff[op], M.FUt[i] + F->ulen[i], nullptr, b, r, 0, b};
          tjb.plane = (size_t)b * M.futcap[i];
          tjb.efix = 1;
          tjb.tld = (int)M.futcap[i];
          usl.push_back(tjb);
        }
        F->ulen[i] += r;
      }
      if (M.mixed) {
        M.FV32[M.k] = f32_alloc(ctx, (int64_t)b * M.Rk);
        c32.push_back(ConvJob{F->Vcol[M.k], M.FV32[M.k], (int64_t)b * M.Rk});
      }
    }
    batched_copy(ctx, cj);
    batched_to_float(ctx, c32);
    oz_split_cols(ctx, usl);
    for (Mat* Mp : L)
      if (Mp->live && Mp->mixed && Mp->nops > 0) panel_tile_norms(ctx, Mp->F, Mp->k, Mp->nL, bnrm);
    pivot_dense_updates(L);
    for (Mat* Mp : L) Mp->stepped = true;
  }
};

void factor_batch(tlr_ctx* ctx, const std::vector<tlr_mat*>& mats_in, const std::vector<double>& eps_in,
                  const std::vector<tlr_opts>& opts, int ldl, std::vector<tlr_status>& status) {
  const int nm = (int)mats_in.size();
  status.assign(nm, TLR_OK);
  if (nm == 0) return;
  Session S(ctx);
  for (int m = 0; m < nm; ++m) S.add(mats_in[m], eps_in[m], opts[m], ldl);
  while (S.busy()) S.step();
  TLR_REQUIRE(!oz_timeout_flag(ctx), TLR_ERR_TIMEOUT, "split product: a bounded device wait ran out");
  for (int m = 0; m < nm; ++m) status[m] = S.status(m);
}

}  // namespace tlr

// ======================================================================== session C ABI
struct tlr_session {
  tlr::Session S;
  std::vector<int> tickets;
  explicit tlr_session(tlr_ctx* c) : S(c) {}
};

#define SESSION_TRY try {
#define SESSION_CATCH                               \
  }                                                 \
  catch (const tlr::Error& e) {                     \
    fprintf(stderr, "[tlr] %s\n", e.what());        \
    return e.status;                                \
  }                                                 \
  catch (...) {                                     \
    return TLR_ERR_CUDA;                            \
  }

extern "C" {

tlr_status tlr_session_create(tlr_ctx* ctx, tlr_session** out) {
  if (!ctx || !out) return TLR_ERR_ARG;
  SESSION_TRY
  *out = new tlr_session(ctx);
  return TLR_OK;
  SESSION_CATCH
}

tlr_status tlr_session_destroy(tlr_session* s) {
  if (!s) return TLR_ERR_ARG;
  SESSION_TRY
  delete s;
  return TLR_OK;
  SESSION_CATCH
}

tlr_status tlr_session_add(tlr_session* s, tlr_mat* A, double eps, const tlr_opts* opts, int ldl, int* ticket) {
  if (!s || !A || !ticket || !(eps > 0)) return TLR_ERR_ARG;
  if (A->state != 0) return TLR_ERR_STATE;
  tlr_opts o;
  if (opts) o = *opts; else tlr_opts_default(&o);
  if (o.bs <= 0) o.bs = 16;
  if (!tlr::factor_opts_ok(o, ldl, A->N, A->b) || (s->S.bs >= 0 && o.bs != s->S.bs)) return TLR_ERR_ARG;
  SESSION_TRY
  *ticket = s->S.add(A, eps, o, ldl);
  return TLR_OK;
  SESSION_CATCH
}

tlr_status tlr_session_step(tlr_session* s, int* unfinished) {
  if (!s) return TLR_ERR_ARG;
  SESSION_TRY
  s->S.step();
  TLR_REQUIRE(!tlr::oz_timeout_flag(s->S.ctx), TLR_ERR_TIMEOUT, "split product: a bounded device wait ran out");
  if (unfinished) {
    int n = 0;
    for (auto& M : s->S.mats) n += (M->live && !M->done) ? 1 : 0;
    *unfinished = n;
  }
  return TLR_OK;
  SESSION_CATCH
}

tlr_status tlr_session_poll(tlr_session* s, int ticket, int* finished, tlr_status* result) {
  if (!s || ticket < 0 || ticket >= (int)s->S.mats.size() || !finished) return TLR_ERR_ARG;
  *finished = s->S.finished(ticket) ? 1 : 0;
  if (result) *result = s->S.status(ticket);
  return TLR_OK;
}

}  // extern "C"
