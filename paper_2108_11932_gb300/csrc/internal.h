// Declarations shared by the host-side translation units of the TLR library.
#pragma once

#include <math.h>

#include <algorithm>
#include <vector>

#include "common.h"

namespace tlr {

// Grow-only device workspace.
struct Buf {
  tlr_ctx* ctx = nullptr;
  void* p = nullptr;
  size_t cap = 0;
  explicit Buf(tlr_ctx* c) : ctx(c) {}
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { dfree(ctx, p); }
  void release() {  // back to empty (the next need() allocates again)
    dfree(ctx, p);
    p = nullptr;
    cap = 0;
  }
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

void d2h_sync(tlr_ctx* ctx, void* host, const void* dev, size_t bytes);

// dense diagonal tiles (blocked, 64-wide blocks)
constexpr int NBK = 64;
struct DenseTile {
  double* A;     // n x n lower, lda
  double* dvec;  // LDL^T: D (n), else null
  int* info;     // device int, -1 on entry
  double* Linv;  // output of the inverse (n x n, ld n), or null
  int n, lda;
};
// workspace (doubles) that dense_factor_batch and dense_trinv_batch take from tmp
size_t dense_tmp_doubles(const std::vector<DenseTile>& tiles, int ldl);
void dense_factor_batch(tlr_ctx* ctx, std::vector<DenseTile>& tiles, int ldl, Buf& tmp);
void dense_trinv_batch(tlr_ctx* ctx, std::vector<DenseTile>& tiles, int unit, Buf& tmp);
void dense_trsm(tlr_ctx* ctx, int n, const double* L, int lda, int unit, int nrhs, double* X, int ldx, int trans);
// Algorithm 8 on a tile that is not positive definite (k_modchol.cu): A (lower triangle read) is replaced
// by the Cholesky factor of A + E (lower; the strict upper triangle holds A + E), Linv (n x n, or null) by
// its inverse, *info (device) by -1 or the failing column of A + E
void modified_cholesky_tile(tlr_ctx* ctx, int n, double* A, int lda, double* Linv, int* info, Buf& work, Buf& tmp);

// ARA engine (Algorithm 1 batched, dynamic batching of Algorithm 5)
struct Sampler {
  virtual ~Sampler() {}
  // true: the sampler draws its own Gaussian blocks (one per matrix of the batch)
  virtual bool owns_omega() const { return false; }
  // Y[s] = T_{ops[s]} Omega_t, written to Ydst[s] (n_op x bs, leading dimension n_op).
  virtual void sample(const std::vector<int>& ops, int t, const double* Om, const std::vector<double*>& Ydst) = 0;
  // B_op = T_op^T Q_op for every operand, given the final widths q.
  virtual void project(const std::vector<int>& q) = 0;
};
struct AraConfig {
  int bs;
  uint64_t seed;      // Gaussian blocks drawn by the engine (when the sampler does not own them)
  uint32_t stream, k;
  int max_slots;
  // every round's orthogonalization in the fused kernel (k_orth.cu).  Otherwise a round whose FP64
  // work exceeds ORTH_FUSED_MAX_FMA runs as batched GEMMs and Cholesky-QR launches, which keep the FP64
  // unit busier on large rounds; the choice depends on the round alone, so it is deterministic for a
  // given input, but a slot's rounding then depends on the slots it shares a round with, which the
  // factorization (whose batches span matrices and sessions) must not allow.
  bool fused_all = false;
};
constexpr double ORTH_FUSED_MAX_FMA = 1.3e8;
struct AraStats {
  int64_t rounds = 0;   // sum over operands of their rounds
  int64_t batches = 0;  // number of batched rounds
  double flops = 0;     // orthogonalization flops (FP64)
};
extern const double HALKO;
extern const double TAU_DROP;

// Fused orthogonalization round (k_orth.cu, block width 16 or 32): for every slot, BCGS2 of its sample block Y against its
// basis Q (n x q, room for q + bs columns) and Cholesky-QR with dropping, in one launch; writes the
// slot's {converged, kept} pair to status[2 s], its new basis columns at Q + q n, uses W as workspace.
struct OrthSlot {
  double* Q;
  double* Y;
  double* W;
  int n, q;
  double thr;
};
bool orth_fused_ok(int bs);
void orth_round(tlr_ctx* ctx, int bs, const std::vector<OrthSlot>& slots, int* status, double* enorm, double tau, Buf& work);
// 1 if a bounded wait of the orthogonalization kernel ran out since the last call (then cleared)
int orth_timeout_flag(tlr_ctx* ctx);
// nrow[op] = rows of operand op; thr[op] = its convergence threshold (eps / HALKO);
// Q_op at Q + qoff[op] with room for nrow[op] x (nrow[op] + bs).
void ara_run(tlr_ctx* ctx, Sampler& S, const std::vector<int>& nrow, const std::vector<double>& thr,
             const AraConfig& cf, const std::vector<int>& order, double* Q, const std::vector<int64_t>& qoff,
             std::vector<int>& q, AraStats& st);

// Uniform dense ARA: nops operands T + op*n*n (n x n); Q (nops x n x (n+bs)), B (nops x n x n).
// BF16 slices of a batch of dense tiles for the split products (k_ozaki.cu)
struct OzTiles {
  int8_t* Sc;  // chunk planes in the tiles' layout (columns of T contiguous)
  int8_t* Sr;  // transposed chunk planes (rows of T contiguous)
  int* e;        // per-tile exponent (device)
  Buf* bx;       // workspace for the right operand's slices
  Buf* be;       // workspace for its column exponents
  double thr8 = 0.0;  // mixed precision: 1/8 of the ARA threshold (0: every product FP64-exact)
};
void ara_dense_run(tlr_ctx* ctx, int nops, int n, const double* T, int bs, double eps, uint64_t seed, uint32_t stream,
                   uint32_t k, double* Q, double* B, std::vector<int>& q, AraStats& st, const OzTiles* oz = nullptr);

// TLR matrix helpers
inline int64_t ix(const tlr_mat* M, int i, int j) { return (int64_t)i * M->nb + j; }
inline double* Uptr(const tlr_mat* M, int i, int j) { return M->Urow[i] + (size_t)M->b * M->uoff[ix(M, i, j)]; }
inline double* Vptr(const tlr_mat* M, int i, int j) { return M->Vcol[j] + (size_t)M->b * M->voff[ix(M, i, j)]; }
void mat_free_storage(tlr_ctx* ctx, tlr_mat* M);
void mat_drop_plans(tlr_ctx* ctx, tlr_mat* M);  // solve plans (and their graphs) of M
void mat_destroy(tlr_ctx* ctx, tlr_mat* M);
tlr_mat* mat_new(int64_t N, int d, int b);
void ensure_ucap(tlr_ctx* ctx, tlr_mat* F, int i, int64_t extra);
// ARA -> SVD rank trimming (k_trim.cu): tile B (b x r, leading dimension b) of a tile Q B^T
struct TrimTile {
  const double* B;
  int r;
};
bool trim_fits(int b);
// ranks r' (host) and, per tile, Z_r (device, r x r', leading dimension r, inside `work`)
void trim_tiles(tlr_ctx* ctx, int b, const std::vector<TrimTile>& tiles, double eps, std::vector<int>& rank,
                std::vector<double*>& Zs, Buf& work);
void trim_matrix(tlr_ctx* ctx, tlr_mat* M, double eps);
// The rules of the factorization options (bs already defaulted), shared by tlr_potrf / tlr_ldlt /
// tlr_factor_batch, tlr_session_add and tlr_submit.
bool factor_opts_ok(const tlr_opts& o, int ldl, int64_t N, int b);

// Batched left-looking TLR Cholesky / LDL^T over several matrices (factor.cu).
// On return status[m] is TLR_OK (mats[m] now holds its factor) or an error
// (TLR_ERR_NOT_SPD: mats[m] in state FAILED with k_fail set).
void factor_batch(tlr_ctx* ctx, const std::vector<tlr_mat*>& mats, const std::vector<double>& eps,
                  const std::vector<tlr_opts>& opts, int ldl, std::vector<tlr_status>& status);

}  // namespace tlr
