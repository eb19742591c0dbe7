// Internal declarations of the GB300 TLR library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <stdexcept>
#include <cstdio>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tlr.h"

namespace tlr {

// Error carried inside the library; converted to a tlr_status at the ABI.
struct Error : std::runtime_error {
  tlr_status status;
  Error(tlr_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TLR_CUDA(x)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      throw ::tlr::Error(TLR_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TLR_REQUIRE(c, st, msg) \
  do {                          \
    if (!(c)) throw ::tlr::Error((st), (msg)); \
  } while (0)

// Launch bookkeeping: every kernel launch of the library goes through this.
#define TLR_LAUNCH_CHECK(ctx) \
  do {                        \
    (ctx)->launches++;        \
    TLR_CUDA(cudaPeekAtLastError()); \
    if ((ctx)->site_out && (ctx)->prof) ::tlr::site_tick((ctx), __FILE__, __LINE__); \
  } while (0)

// Ω streams: which factorization step a Gaussian block belongs to.
enum : uint32_t { STREAM_COMPRESS = 1, STREAM_FACTOR = 2, STREAM_SCHUR = 3 };

// Column-major batched GEMM job: C(M x N) = alpha * sum_s op(A_s) op(B_s) + beta * C.
// op(A_s) is M x K_s, op(B_s) is K_s x N.  Up to two K-segments (the products
// "[U0 | Urow] W" of the sampling chain have two left operands).
template <typename T>
struct GemmJob {
  const T* A[2];
  const T* B[2];
  T* C;
  T* ws;         // split-K partials: nsplit x M x N (column-major), or null
  int* ctr;      // split-K: arrival counter per output tile (tiles_m x tiles_n)
  int lda[2], ldb[2], K[2];
  int ldc, M, N;
  int tile0;     // first linear CTA of this job
  int tiles_m, tiles_n, nsplit;
  int flags;     // GEMM_TRIL: write only C(m, n) with m >= n; skip tiles strictly above
                 // GEMM_ALOWER: op(A_0) is lower triangular (NN only): row m reads k <= m
  int rule_n;    // columns the split-K rule assumes (0: N), so that a product formed for several
                 // right-hand blocks at once sums every element as the one-block product does
  double alpha, beta;
};
enum { GEMM_TRIL = 1, GEMM_ALOWER = 2 };
enum GemmMode { NN = 0, TN = 1, NT = 2 };

constexpr int GEMM_TK = 16;

}  // namespace tlr

namespace tlr {
struct SolvePlan;
struct Server;
}

// ----------------------------------------------------------------------------------------
// Library-owned objects.
struct tlr_ctx {
  int device = 0;
  // device bytes this context holds (every allocation goes through dalloc / dfree) and the serving
  // queue's admission budget (tlr_create's hbm_budget; 0 = no limit)
  size_t hbm_budget = 0;
  size_t live_bytes = 0, peak_bytes = 0;
  std::unordered_map<void*, size_t> live;
  tlr::Server* server = nullptr;  // request queue of tlr_submit / tlr_progress / tlr_poll (serve.cu)
  cudaStream_t stream = nullptr;  // stream the next launch goes to (main or side)
  cudaStream_t main = nullptr;    // caller's stream
  cudaStream_t side = nullptr;    // library stream for work overlapped with the main stream
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t capture = nullptr;  // library stream on which solve graphs are captured
  tlr_alloc_fn alloc = nullptr;
  tlr_free_fn free_fn = nullptr;
  void* user = nullptr;
  int sm_count = 0;
  int64_t launches = 0;
  // Job upload ring: pinned host staging mirrored by a device buffer.
  char* pinned = nullptr;
  char* djobs = nullptr;
  size_t ring_cap = 0, ring_pos = 0;
  // Split-K / small scratch, grown on demand (stream-ordered frees).
  void* scratch = nullptr;
  size_t scratch_cap = 0;
  void* scratch_side = nullptr;  // the side stream's own split-K scratch
  size_t scratch_side_cap = 0;
  // split-K arrival counters (zero between launches; the reducing CTA resets its
  // own), one array per stream
  int* split_ctr[2] = {nullptr, nullptr};
  size_t split_ctr_cap[2] = {0, 0};
  // grid-barrier words of the fused orthogonalization kernel: {arrivals, generation} per stream
  unsigned* orth_bar = nullptr;
  // Small host-pinned status buffer for per-round device->host reads.
  void* hstatus = nullptr;
  size_t hstatus_cap = 0;
  // Phase profiler (CUDA events at phase boundaries; off by default).
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_phase;
  size_t ev_n = 0;
  double phase_ms[16] = {0};
  int64_t phase_launch[16] = {0};
  int cur_phase = -1;
  int64_t phase_launch0 = 0;
  double host_wait_ms = 0;  // host time blocked in stream synchronizations while profiling
  // Per-kernel accounting of the batched GEMM launches (CUDA events around each launch).
  bool kprof = false;
  std::vector<cudaEvent_t> kev;
  std::vector<int> kev_fam;
  std::vector<double> kev_flops, kev_bytes;
  size_t kev_n = 0;
  double kfam_ms[8] = {0}, kfam_flops[8] = {0}, kfam_bytes[8] = {0};
  int64_t kfam_launches[8] = {0};
  // Per-call-site launch profile (diagnostics): while tlr_profile is enabled and the
  // TLR_SITE_PROFILE environment variable names a file, which receives the table at
  // tlr_destroy.  An
  // event follows every launch; a launch is charged the time between the previous
  // event of its stream and its own, i.e. its device time while the stream is busy.
  FILE* site_out = nullptr;
  std::vector<cudaEvent_t> sev[2];
  std::vector<int> sev_site[2];
  size_t sev_n[2] = {0, 0};
  std::map<std::pair<const char*, int>, int> site_id;
  std::vector<std::string> site_name;
  std::vector<double> site_ms;
  std::vector<int64_t> site_count;
  std::vector<double> site_flops;   // algorithmic flops of the site's launches (GEMMs)
  std::vector<double> sev_flops[2];
  double site_next_flops = 0;       // set by a launcher just before its launch is ticked
};

struct tlr_mat {
  int64_t N = 0;
  int d = 0, b = 0, nb = 0;
  int state = 0;  // 0 A, 1 chol, 2 ldlt, 3 failed
  int k_fail = -1;
  tlr_kernel kern{};
  double eps = 0;
  std::vector<int64_t> perm;
  double* pts = nullptr;   // device, ordered points (N x d row-major)
  int64_t* dperm = nullptr;  // device copy of perm
  double* diag = nullptr;  // device, nb * b * b
  double* dvec = nullptr;  // device, nb * b (LDL^T D)
  double* dinv = nullptr;  // device, nb * b * b: inverses of the (unit for LDL^T) lower diagonal tiles
  std::vector<int> rank;   // nb * nb (i > j)
  std::vector<int64_t> uoff, voff;  // column offsets of U_ij in Urow[i], V_ij in Vcol[j]
  std::vector<double*> Urow, Vcol;  // per block row / block column panels (device)
  std::vector<int64_t> ucap;        // capacity (columns) of Urow[i]
  std::vector<int64_t> vlen;        // columns of Vcol[j]
  std::vector<int64_t> ulen;        // used columns of Urow[i]
  // statistics of the last factorization
  double flops_exec = 0, flops_model = 0, ara_rounds = 0, seconds = 0;
  double tiles_fp32 = 0, tiles_fp64 = 0;  // tile-rounds sampled in each precision (mixed mode)
  double flops_fp32 = 0;                  // FP32 flops of the mixed-precision chains
  // solve plans of a factor (buffers, job tables, captured graph), one per nrhs, most recent last
  std::vector<tlr::SolvePlan*> plans;
};

namespace tlr {

// phase profiler: the stream time between two marks is charged to the first mark's phase
enum Phase { PH_GRAM = 0, PH_DIAG, PH_POTRF, PH_SAMPLE, PH_ORTH, PH_SYNC, PH_PROJECT, PH_TRSM, PH_UPDATE,
             PH_COMPRESS, PH_SOLVE, PH_OTHER, PH_COUNT };
void prof_mark(tlr_ctx* ctx, int phase);
void prof_flush(tlr_ctx* ctx);
// kernel families of the GEMM accounting: fp64 NN/TN/NT, fp32 NN/TN/NT
void kprof_begin(tlr_ctx* ctx);
// families: 0-2 FP64 k_gemm NN/TN/NT, 3-5 FP32 k_gemm, 6 split products (k_oz_mma), 7 k_orth_round
void kprof_end(tlr_ctx* ctx, int family, double flops, double bytes = 0);
void kprof_flush(tlr_ctx* ctx);
void site_tick(tlr_ctx* ctx, const char* file, int line);
// an event just before a launch: the time since the stream's previous event is
// charged to "gaps" (copies, waits, host delays), so that the launch's own site
// receives its device time only
#define TLR_SITE_PRE(ctx) \
  do {                    \
    if ((ctx)->site_out && (ctx)->prof) ::tlr::site_tick_on((ctx), (ctx)->stream, nullptr, 0); \
  } while (0)
// marks the end of a wait (event wait, host synchronization) on a stream
void site_tick_on(tlr_ctx* ctx, cudaStream_t stream, const char* file, int line);
#define TLR_SITE_MARK(ctx, stream) \
  do {                                \
    if ((ctx)->site_out && (ctx)->prof) ::tlr::site_tick_on((ctx), (stream), __FILE__, __LINE__); \
  } while (0)
void site_flush(tlr_ctx* ctx);
void site_report(tlr_ctx* ctx);

// memory
void server_destroy(tlr_ctx* ctx);  // serve.cu: frees every request still held
void* dalloc(tlr_ctx* ctx, size_t bytes);
void dfree(tlr_ctx* ctx, void* p);
void* scratch(tlr_ctx* ctx, size_t bytes);
// zeroed split-K arrival counters for the current stream (at least n)
int* split_counters(tlr_ctx* ctx, size_t n);
void* upload(tlr_ctx* ctx, const void* host, size_t bytes);  // returns device copy (ring)
void* host_status(tlr_ctx* ctx, size_t bytes);               // pinned host buffer

// GEMM (k_gemm.cu)
template <typename T>
void gemm(tlr_ctx* ctx, GemmMode mode, std::vector<GemmJob<T>>& jobs);
template <typename T>
GemmJob<T> job(GemmMode mode, int M, int N, const T* A, int lda, const T* B, int ldb, int K, T* C,
               int ldc, double alpha, double beta);

// Kernels (k_misc.cu) -- all enqueue on ctx->stream.
void omega(tlr_ctx* ctx, uint64_t seed, uint32_t stream, uint32_t k, uint32_t t, int b, int bs,
           double* out);
// Points on a 64-bit grid for the kernel tiles: X (device, N x d) = round(x 2^q) - round(o 2^q).
struct GridInfo {
  int q;
  int pad;
  double o[3];
};
void grid_points(tlr_ctx* ctx, const double* pts, int64_t N, int d, GridInfo* gi /*device*/, long long* X);
void gen_tiles(tlr_ctx* ctx, const long long* X, const GridInfo* gi, int64_t N, int d, double ell, double nugget,
               int b, const int* tile_ij /*device, 2 per tile*/, int ntiles, double* out,
               unsigned long long* tmax = nullptr /*device, per tile, zeroed*/);
// per-slot orthogonalization helpers (Cholesky-QR with dropping)
// thr: device array, per-slot convergence threshold
void cholqr_small(tlr_ctx* ctx, int nslots, int bs, const double* G, double* Mout, int* status,
                  double* enorm, const double* thr, double tau, int first_pass, const int* nk_in);
// dense diagonal-tile factorization pieces (batched over tiles; the single-tile forms wrap them)
struct PotrfJob {
  double* A;
  double* dvec;  // LDL^T: D of the whole tile (entries col0.. written)
  int* info;
  double* Binv;  // receives the inverse of the factored block (lower; zeros above), ld ldb
  int lda, col0, nbk, ldb;
};
struct PanelJob {
  const double* Binv;  // inverse of the factored diagonal block (lower), ld ldb
  double* X;           // panel below the block, m x nbk, updated in place
  const double* dvec;  // LDL^T: D of this block
  double* W;           // LDL^T: receives X L^{-T} before the D^{-1} scaling (m x nbk, ld m)
  int ldb, ldx, m, nbk;
};
struct LeftJob {
  const double* L;
  double* X;
  int lda, ldx, nrhs, nbk;
};
void potrf_inv_blocks(tlr_ctx* ctx, std::vector<PotrfJob>& jobs, int ldl);
void panel_apply(tlr_ctx* ctx, std::vector<PanelJob>& jobs, int ldl);
void trsm_lefts(tlr_ctx* ctx, std::vector<LeftJob>& jobs, int unit, int trans);
void trsm_left_block(tlr_ctx* ctx, int nbk, const double* L, int lda, int unit, int nrhs, double* X,
                     int ldx);
void trsm_left_t_block(tlr_ctx* ctx, int nbk, const double* L, int lda, int unit, int nrhs,
                       double* X, int ldx);
void scale_rows(tlr_ctx* ctx, int m, int n, const double* dvec, int inv, const double* X, int ldx,
                double* Y, int ldy);
void add_diag(tlr_ctx* ctx, int n, double* A, int lda, double s);
void add_rowsum_abs(tlr_ctx* ctx, int n, const double* E, int lde, double* A, int lda);
void logdet_reduce(tlr_ctx* ctx, int n, const double* diag_tiles, int b, int nb, const double* dvec,
                   double* out2 /*device: [sum log|.|, count negative]*/);
void kernel_matvec(tlr_ctx* ctx, const double* pts, int64_t N, int d, double ell, double nugget,
                   int nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy);
void permute_rows(tlr_ctx* ctx, int64_t n_out, int nrhs, const int64_t* idx, int gather,
                  const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t n_pad);
void copy_matrix(tlr_ctx* ctx, int m, int n, const double* X, int ldx, double* Y, int ldy);
void to_float(tlr_ctx* ctx, int64_t n, const double* x, float* y);
void to_double(tlr_ctx* ctx, int64_t n, const float* x, double* y);

// blocked chains of the sampling (k_misc.cu): see the definitions for layouts.
template <typename T>
struct SlotDescT {
  const int* rank;   // the slot's matrix: ranks, U / V column offsets (nb x nb, device)
  const int* uoff;
  const int* voff;
  const int64_t* goff;  // Gram blocks of the matrix's current column
  const int* gld;
  const T* G;
  const T* X;        // sample: X = Urow_k^T Omega (Kk x bs), X0 = V0col_k^T Omega
  const T* X0;
  T* W;              // sample output block ((r0 + Ki) x bs)
  T* P;              // project: P block ((r0 + Ki) x q) and output Z ((r0 + Kk) x q)
  T* Z;
  int ldx, ldx0, nb, k, i, r0, x0off, Ki, Kk, q, bs;
  int r0w;           // sample: rows of W holding X0 (r0, or r0 rounded up to 32 and zero-padded when the
                     // product runs as one split product over [U0 | Urow])
};
// FP64 products on the 16-bit tensor cores by exact splitting (k_ozaki.cu).  Operands are stored as 8
// planes of signed 7-bit chunks (int8, one byte per chunk); rows of a plane start on 16-byte
// boundaries (the TMA rule), so leading dimensions along k are padded to oz_ld(K).
inline __host__ __device__ int oz_ld(int K) { return (K + 15) / 16 * 16; }
// columns to split: X (K x ncols, ld) -> plane q of column c at Xs + q * plane + c * ldo (rows
// K .. ldo-1 zero), relative to 2^e[c] (e[c] computed), or to 2^efix for every column
constexpr int OZ_EFIX_NONE = -100000;
struct OzColJob {
  const double* X;
  int8_t* Xs;
  int* e;
  int ld, ncols, col0, K;
  size_t plane = 0;  // 0: ncols * ldo
  int ldo = 0;       // 0: oz_ld(K)
  int efix = OZ_EFIX_NONE;
  // with emax (device: the block's largest |x| as FP64 bits) every column uses that block bound,
  // written to e[0]
  const unsigned long long* emax = nullptr;
  // tld > 0: transposed output, element k of column c at Xs + q * plane + k * tld + c (k < K only)
  int tld = 0;
};
// C (M x N, ldc) = A B (or C += A B), A(m, k) = A_q[k + m * lda] (rows along k) or, with acol,
// A_q[m + k * lda] (columns along m); B(k, n) = B_q[k + n * ldb].  lda, ldb, the plane strides and
// the operand addresses are multiples of 16 bytes.
struct OzJob {
  const int8_t* A;       // 8 chunk planes, stride sA (bytes)
  const int8_t* B;       // 8 chunk planes, stride sB
  const int* eA;         // block exponent of A (device)
  const int* eB;         // column exponents of B (device, N)
  double* C;
  size_t sA, sB;
  int lda, ldc, M, N, K;
  int ldb = 0;           // 0: oz_ld(K)
  int acol = 0;
  int accumulate = 0;
  int eB_stride = 1;     // 0: one exponent for all columns of B
  // split K: slices of whole 32-deep stages, FP64 partials in ws, summed in slice order by the
  // last CTA of each output block (arrival counters).  nsplit = 0 lets oz_gemm choose from the
  // job's shape; the caller may fix it (1: no split).
  int nsplit = 0, tiles_n = 1;
  int rule_n = 0;        // columns the split rule assumes (0: N), as for GemmJob
  int S = 8;             // chunk planes used (8: FP64-exact; fewer: both operands truncated to 7S bits)
  // mixed precision: with tol > 0 each CTA uses the fewest planes s >= smin (at most S) whose error
  // bound per entry, K (s + 1) 2^(eA + eB - 7 s), stays below tol (an absolute error)
  double tol = 0.0;
  int smin = 2;
  // optional first K segment (rows along k, not acol): A(m, k) for k < K0 from A0 (8 planes, stride
  // sA0, leading dimension lda0), A(m, k) = A_q[(k - K0) + m * lda] for k >= K0; K0 a multiple of 32,
  // the segment zero past its data; both segments relative to the block exponent eA
  const int8_t* A0 = nullptr;
  size_t sA0 = 0;
  int lda0 = 0, K0 = 0;
  double* ws = nullptr;
  int* ctr = nullptr;
};
// Sc may be null (only the transposed chunks are written)
void oz_split_tiles(tlr_ctx* ctx, int ntiles, int n, const double* T, const unsigned long long* tmax, int8_t* Sc,
                    int8_t* Sr, int* eT);
void oz_split_cols(tlr_ctx* ctx, std::vector<OzColJob>& jobs);
void oz_absmax(tlr_ctx* ctx, int nblocks, int64_t n2, const double* T, unsigned long long* tmax);
void oz_gemm(tlr_ctx* ctx, std::vector<OzJob>& jobs);
// Synchronizes the stream and returns (and clears) the flag a split product sets when one of its
// bounded waits ran out.
int oz_timeout_flag(tlr_ctx* ctx);
// CTAs of the split products by planes used (out[1..8]) and chunk bytes read (out[9]), since the
// last reset
void oz_stats(tlr_ctx* ctx, unsigned long long out[10], int reset);

// one 16 x 16 output tile of a block-diagonal Gram product: slot, block column j
// (j = k: the tile's own factor part), row chunk, column chunk
struct BlkItem {
  uint32_t slot;
  uint16_t j;
  uint8_t rc, cc;  // ranks and widths are at most 1024: 64 chunks
};
template <typename T>
void blkdiag_sample(tlr_ctx* ctx, const std::vector<BlkItem>& items, const SlotDescT<T>* slots_dev);
template <typename T>
void blkdiag_project(tlr_ctx* ctx, const std::vector<BlkItem>& items, const SlotDescT<T>* slots_dev);

struct OmegaJob {
  double* out;
  uint64_t seed;
  uint32_t stream, k, t;
  int b, bs;
};
void omega_batched(tlr_ctx* ctx, std::vector<OmegaJob>& jobs);
struct ConvBackJob {
  const float* src;
  double* dst;
  int64_t n;
};
void batched_to_double(tlr_ctx* ctx, std::vector<ConvBackJob>& jobs);
struct ScaleJob {
  const double* d;
  const double* X;
  double* Y;
  int m, n, ldx, ldy, inv;
};
void batched_scale_rows(tlr_ctx* ctx, std::vector<ScaleJob>& jobs);
struct DiagJob {
  double* A;
  int n, lda;
  double s;
};
void batched_add_diag(tlr_ctx* ctx, std::vector<DiagJob>& jobs);

double fp64_peak(tlr_ctx* ctx);

struct CopyJob {
  const double* src;
  double* dst;
  int64_t n;
};
void batched_copy(tlr_ctx* ctx, std::vector<CopyJob>& jobs);
// Skinny products of the triangular solves (k_solve.cu): C = alpha op(A) B + beta C with nrhs
// columns, op(A) = A (tn = 0, A M x K) or A^T (tn = 1, A K x M), all column-major; lower: A is a
// lower-triangular block (its zero half is skipped).  Job tables are device-resident.
struct SkJob {
  const double* A;
  const double* B;
  double* C;
  int lda, ldb, ldc, M, K, lower;
  double alpha, beta;
};
// work items of a launch: one CTA each (job, first row, log2 of the k-slots of an NN product)
struct SkItem {
  int job, m0, cfg;
};
void sk_items(int tn, const std::vector<SkJob>& jobs, int job0, std::vector<SkItem>& items);
void sk_gemm(tlr_ctx* ctx, int tn, const SkJob* jobs, const SkItem* items, int nitems, int nrhs);
// Preconditioned CG vectors (k_solve.cu): per-column dot products (fixed-order sums) and the two
// vector updates of an iteration, with per-column coefficients num/den read on the device.
void coldot(tlr_ctx* ctx, int64_t n, int ncols, const double* X, int64_t ldx, const double* Y, int64_t ldy,
            double* out);
void pcg_update_xr(tlr_ctx* ctx, int64_t n, int ncols, const double* num, const double* den, const int* active,
                   double* x, int64_t ldx, const double* p, double* r, const double* q, int64_t ld);
void pcg_update_p(tlr_ctx* ctx, int64_t n, int ncols, const double* num, const double* den, const int* active,
                  const double* z, double* p, int64_t ld);
struct ConvJob {
  const double* src;
  float* dst;
  int64_t n;
};
void batched_to_float(tlr_ctx* ctx, std::vector<ConvJob>& jobs);
void col_sqnorms(tlr_ctx* ctx, const double* X, int rows, int64_t ncols, double* out);
void scale_cols(tlr_ctx* ctx, int m, int n, const double* dvec, const double* X, int ldx, double* Y,
                int ldy);
void tril_mask(tlr_ctx* ctx, int n, double* A, int lda, int unit);
void set_diag(tlr_ctx* ctx, int n, double* A, int lda, const double* d);
void axpy_matrix(tlr_ctx* ctx, int m, int n, double alpha, const double* X, int ldx, double* Y, int ldy);

// Argument rule shared by tlr_kernel_matvec and tlr_kernel_matvec_noalloc (the same Y = A X): the
// exponential kernel with ell > 0 and nugget >= 0, 1 <= d <= 3, N > 0, nrhs >= 0, ldx, ldy >= N.
inline bool kernel_product_args_ok(const double* pts, const tlr_kernel* k, const double* X, const double* Y, int64_t N,
                                   int d, int nrhs, int64_t ldx, int64_t ldy) {
  return pts && k && X && Y && N > 0 && d >= 1 && d <= 3 && nrhs >= 0 && ldx >= N && ldy >= N && k->ell > 0 &&
         k->type == TLR_KERNEL_EXP && k->nugget > -1.0;
}

// kdtree.cpp
void kd_order(const double* pts, int64_t N, int d, int b, int64_t* perm);

}  // namespace tlr
