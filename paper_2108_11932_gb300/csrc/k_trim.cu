// ARA -> SVD rank trimming of low-rank tiles (Section 6: the post-processing step that applies the SVD
// to each low-rank tile to bring its rank down to the minimum).
//
// A tile Q B^T with orthonormal Q (b x r) has the singular values of B.  One CTA per tile: a Householder
// QR of B (B = H R, the reflectors applied to the trailing columns in place, in a working copy in global
// memory: the QR runs at GB300's FP64 rate, and a small shared footprint lets several tiles share an SM),
// then one-sided Jacobi (Hestenes) on X = R^T: plane rotations of column pairs in the parallel
// round-robin order (r/2 disjoint pairs per round, r - 1 rounds per sweep) until no pair is rotated,
// giving X J = Y with orthogonal columns whose norms are the singular values sigma of R (and of B), and
// Y / sigma the right singular vectors Z of B (R = J S (Y S^-1)^T).  Jacobi on R^T rather than R takes
// about a third of the sweeps on these matrices.  The columns with sigma > eps, in descending order,
// form Z_r (r x r'); Q' = Q Z_r and B' = B Z_r = W_r S_r are two batched GEMMs.  Every reduction has a
// fixed order, so the result depends on the tile only.
#include <math.h>

#include <map>

#include "internal.h"

namespace tlr {

namespace {

constexpr int TR_T = 256, TR_W = TR_T / 32;
constexpr int TR_SWEEPS = 60;  // a bound only: the tiles converge in about 10

struct TrimDev {
  const double* B;  // b x r, leading dimension b
  double* W;        // working copy (b x r)
  double* X;        // R^T (r x r) when it does not live in shared memory
  double* Zs;       // out: Z_r (r x r', leading dimension r)
  int* rank;        // out: r'
  int r;
};

// warp sum, the lane-0 value broadcast so that every lane holds the same bits
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();  // red is free
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < TR_W; ++i) s += red[i];
  return s;
}

// MODE 0: X = R^T in global memory; 1: X in shared memory (after the reflector vector, the singular
// values and their order)
template <int MODE>
__global__ void __launch_bounds__(TR_T) k_trim(const TrimDev* __restrict__ jobs, int b, double eps) {
  const TrimDev J = jobs[blockIdx.x];
  const int r = J.r, tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  extern __shared__ double sm[];
  double* v = sm;                                  // b: the current reflector
  double* red = v + b;                             // TR_W
  double* sig = red + TR_W;                        // r
  int* pos = reinterpret_cast<int*>(sig + r);      // r
  double* nxt = reinterpret_cast<double*>(pos + r + (r & 1));
  const int rp = r | 1;  // X's leading dimension, odd: the pair threads below read distinct banks
  double* X = MODE == 1 ? nxt : J.X;
  double* W = J.W;
  __shared__ int rot, keep;
  if (r == 0) {
    if (tid == 0) *J.rank = 0;
    return;
  }
  for (int64_t e = tid; e < (int64_t)b * r; e += TR_T) W[e] = J.B[e];
  __syncthreads();
  // ---- Householder QR: R in the upper triangle of W's first r rows
  for (int j = 0; j < r; ++j) {
    double* cj = W + (size_t)j * b;
    double s = 0.0;
    for (int m = j + 1 + tid; m < b; m += TR_T) s += cj[m] * cj[m];
    s = block_sum(s, red);
    if (s > 0.0) {  // uniform: s is the block's sum
      const double alpha = cj[j];
      const double nrm = sqrt(alpha * alpha + s);
      const double beta = alpha >= 0.0 ? -nrm : nrm;
      const double tau = (beta - alpha) / beta, scal = 1.0 / (alpha - beta);
      for (int m = j + 1 + tid; m < b; m += TR_T) v[m] = cj[m] * scal;
      if (tid == 0) v[j] = 1.0;
      __syncthreads();  // v complete; every thread has read alpha
      if (tid == 0) cj[j] = beta;
      for (int c = j + 1 + w; c < r; c += TR_W) {  // H = I - tau v v^T on the trailing columns
        double* col = W + (size_t)c * b;
        double d = 0.0;
#pragma unroll 4
        for (int m = j + l; m < b; m += 32) d += v[m] * col[m];
        const double f = tau * warp_sum(d);
#pragma unroll 4
        for (int m = j + l; m < b; m += 32) col[m] -= f * v[m];
      }
    }
    __syncthreads();
  }
  // ---- X = R^T (lower triangular)
  for (int64_t e = tid; e < (int64_t)r * r; e += TR_T) {
    const int m = (int)(e % r), c = (int)(e / r);
    X[m + (size_t)c * rp] = c <= m ? W[c + (size_t)m * b] : 0.0;
  }
  __syncthreads();
  // ---- one-sided Jacobi on X, round-robin pairs (position 0 fixed, 1 .. n-1 rotating), one thread per
  // pair: GB300's FP64 unit is the bound, and a thread's serial dot products waste no lanes on reductions
  const int n = r + (r & 1);
  const double tol = (double)r * 0x1p-53;
  for (int sweep = 0; sweep < TR_SWEEPS; ++sweep) {
    if (tid == 0) rot = 0;
    __syncthreads();
    for (int t = 0; t < n - 1; ++t) {
      for (int k = tid; k < n / 2; k += TR_T) {
        int p = k == 0 ? 0 : (k - 1 + t) % (n - 1) + 1;
        int q = (n - 2 - k + t) % (n - 1) + 1;  // the position n - 1 - k >= 1
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        if (q >= r) continue;  // the padding index of an odd r
        double* xp = X + (size_t)p * rp;
        double* xq = X + (size_t)q * rp;
        double a = 0.0, bb = 0.0, g = 0.0;
        for (int m = 0; m < r; ++m) {
          const double x = xp[m], y = xq[m];
          a = fma(x, x, a);
          bb = fma(y, y, bb);
          g = fma(x, y, g);
        }
        if (g != 0.0 && fabs(g) > tol * sqrt(a * bb)) {
          const double z = (bb - a) / (2.0 * g);
          const double tt = fabs(z) < 1e150 ? (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z)) : 0.5 / z;
          const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
          for (int m = 0; m < r; ++m) {
            const double x = xp[m], y = xq[m];
            xp[m] = c * x - sn * y;
            xq[m] = sn * x + c * y;
          }
          rot = 1;
        }
      }
      __syncthreads();
    }
    if (rot == 0) break;  // read by every thread after the round's barrier
    __syncthreads();      // before thread 0 clears it
  }
  // ---- singular values, their descending order, the kept columns
  for (int c = w; c < r; c += TR_W) {
    const double* xc = X + (size_t)c * rp;
    double s2 = 0.0;
    for (int m = l; m < r; m += 32) s2 += xc[m] * xc[m];
    s2 = warp_sum(s2);
    if (l == 0) sig[c] = sqrt(s2);
  }
  __syncthreads();
  for (int c = tid; c < r; c += TR_T) {
    const double sc = sig[c];
    int ps = 0;
    for (int d = 0; d < r; ++d) ps += (sig[d] > sc || (sig[d] == sc && d < c)) ? 1 : 0;
    pos[c] = ps;
  }
  if (tid == 0) {
    int kk = 0;
    for (int c = 0; c < r; ++c) kk += sig[c] > eps ? 1 : 0;
    keep = kk;
  }
  __syncthreads();
  for (int c = w; c < r; c += TR_W) {
    const int ps = pos[c];
    if (ps >= keep) continue;
    const double inv = 1.0 / sig[c];
    const double* xc = X + (size_t)c * rp;
    double* zc = J.Zs + (size_t)ps * r;
    for (int m = l; m < r; m += 32) zc[m] = xc[m] * inv;
  }
  if (tid == 0) *J.rank = keep;
}

size_t trim_smem(int b, int r, int mode) {
  return sizeof(double) * ((size_t)b + TR_W + r) + sizeof(int) * ((size_t)r + (r & 1)) +
         (mode == 1 ? sizeof(double) * (size_t)r * (r | 1) : 0);
}

constexpr size_t TRIM_SMEM_MAX = 220 * 1024;

}  // namespace

bool trim_fits(int b) { return trim_smem(b, b, 0) <= TRIM_SMEM_MAX; }

void trim_tiles(tlr_ctx* ctx, int b, const std::vector<TrimTile>& tiles, double eps, std::vector<int>& rank,
                std::vector<double*>& Zs, Buf& work) {
  const int nt = (int)tiles.size();
  rank.assign(nt, 0);
  Zs.assign(nt, nullptr);
  if (nt == 0) return;
  TLR_REQUIRE(trim_fits(b), TLR_ERR_LIMIT, "rank trimming: tile size above the shared-memory limit");
  // workspace per tile: W (b r), X (r (r | 1), used when it does not fit in shared memory), Zs (r^2); ranks
  int64_t tot = 0;
  std::vector<int64_t> off(nt);
  for (int t = 0; t < nt; ++t) {
    off[t] = tot;
    tot += (int64_t)tiles[t].r * (b + (tiles[t].r | 1) + (int64_t)tiles[t].r);
  }
  double* ws = work.need<double>((size_t)std::max<int64_t>(tot, 1) + (size_t)(nt + 1) / 2 + 1);
  int* dr = reinterpret_cast<int*>(ws + std::max<int64_t>(tot, 1));
  // launch groups: the most on-chip mode the tile's rank allows, then rank classes (so that a group's
  // shared memory, sized by its largest rank, does not hold many small tiles to one CTA per SM)
  static const int cls[] = {8, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1 << 30};
  std::map<std::pair<int, int>, std::vector<TrimDev>> groups;
  for (int t = 0; t < nt; ++t) {
    const int r = tiles[t].r;
    double* W = ws + off[t];
    double* X = W + (size_t)b * r;
    TrimDev d{tiles[t].B, W, X, X + (size_t)r * (r | 1), dr + t, r};
    Zs[t] = d.Zs;
    const int mode = trim_smem(b, r, 1) <= TRIM_SMEM_MAX ? 1 : 0;
    int c = 0;
    while (cls[c] < r) ++c;
    groups[{mode, c}].push_back(d);
  }
  for (auto& g : groups) {
    const int mode = g.first.first;
    std::vector<TrimDev>& js = g.second;
    int rmax = 0;
    for (const TrimDev& d : js) rmax = std::max(rmax, d.r);
    const size_t sm = trim_smem(b, rmax, mode);
    auto kern = mode == 1 ? k_trim<1> : k_trim<0>;
    if (sm > 48 * 1024) TLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    for (size_t o = 0; o < js.size(); o += 65535) {
      const int cnt = (int)std::min<size_t>(65535, js.size() - o);
      const TrimDev* dj = static_cast<const TrimDev*>(upload(ctx, js.data() + o, sizeof(TrimDev) * cnt));
      TLR_SITE_PRE(ctx);
      kern<<<cnt, TR_T, sm, ctx->stream>>>(dj, b, eps);
      TLR_LAUNCH_CHECK(ctx);
    }
  }
  TLR_CUDA(cudaMemcpyAsync(rank.data(), dr, sizeof(int) * nt, cudaMemcpyDeviceToHost, ctx->stream));
  TLR_CUDA(cudaStreamSynchronize(ctx->stream));
}

// Every off-diagonal tile U_ij V_ij^T of M replaced by Q' B'^T: new block-row and block-column panels
// (ranks never grow), solve plans dropped (they point into the old panels).
void trim_matrix(tlr_ctx* ctx, tlr_mat* M, double eps) {
  const int nb = M->nb, b = M->b;
  std::vector<TrimTile> tl;
  std::vector<std::pair<int, int>> ij;
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < i; ++j) {
      const int r = M->rank[ix(M, i, j)];
      if (r == 0) continue;
      tl.push_back(TrimTile{Vptr(M, i, j), r});
      ij.push_back({i, j});
    }
  Buf work(ctx);
  std::vector<int> rk;
  std::vector<double*> Zs;
  trim_tiles(ctx, b, tl, eps, rk, Zs, work);
  std::vector<int> nr((size_t)nb * nb, 0);
  for (size_t t = 0; t < tl.size(); ++t) nr[ix(M, ij[t].first, ij[t].second)] = rk[t];
  std::vector<double*> Urow(nb, nullptr), Vcol(nb, nullptr);
  std::vector<int64_t> ulen(nb, 0), vlen(nb, 0), uoff((size_t)nb * nb, 0), voff((size_t)nb * nb, 0);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < i; ++j) {
      uoff[ix(M, i, j)] = ulen[i];
      ulen[i] += nr[ix(M, i, j)];
    }
  for (int j = 0; j < nb; ++j)
    for (int i = j + 1; i < nb; ++i) {
      voff[ix(M, i, j)] = vlen[j];
      vlen[j] += nr[ix(M, i, j)];
    }
  for (int i = 0; i < nb; ++i) {
    Urow[i] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(ulen[i], 1) * b));
    Vcol[i] = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(vlen[i], 1) * b));
  }
  std::vector<GemmJob<double>> jobs;
  for (size_t t = 0; t < tl.size(); ++t) {
    const int i = ij[t].first, j = ij[t].second, r = tl[t].r, q = rk[t];
    if (q == 0) continue;
    jobs.push_back(job<double>(NN, b, q, Uptr(M, i, j), b, Zs[t], r, r, Urow[i] + (size_t)b * uoff[ix(M, i, j)], b,
                               1.0, 0.0));
    jobs.push_back(job<double>(NN, b, q, Vptr(M, i, j), b, Zs[t], r, r, Vcol[j] + (size_t)b * voff[ix(M, i, j)], b,
                               1.0, 0.0));
  }
  gemm<double>(ctx, NN, jobs);
  mat_free_storage(ctx, M);  // also drops the solve plans
  M->Urow = Urow;
  M->Vcol = Vcol;
  M->rank = nr;
  M->uoff = uoff;
  M->voff = voff;
  M->ulen = ulen;
  M->vlen = vlen;
  for (int i = 0; i < nb; ++i) M->ucap[i] = std::max<int64_t>(ulen[i], 1);
}

}  // namespace tlr
