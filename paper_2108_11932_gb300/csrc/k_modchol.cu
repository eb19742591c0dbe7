// Modified Cholesky of a diagonal tile (Algorithm 8, Section 5.1.2).
//
// A tile A (n x n, symmetric, lower triangle read) whose Cholesky factorization failed is factored by
// symmetric pivoting, P^T A P = L D L^T with 1x1 and 2x2 pivot blocks chosen by the partial pivoting
// rule of Bunch and Kaufman (1977) (alpha = (1 + sqrt 17) / 8, the first largest entry on ties, the
// updates of the unblocked LAPACK form).  Each pivot block's eigenvalues are then raised to at least
// delta = sqrt(u / 2) ||A||_inf (the choice of Cheng and Higham, 1998), giving D + F positive
// definite, and the tile is replaced by A + E = P L (D + F) L^T P^T, symmetrized, whose Cholesky factor
// the caller takes.  One CTA runs the pivoted factorization (a dependent sequence of n steps over the
// trailing matrix, in global memory); the reconstruction is a batched GEMM.
#include <math.h>

#include "internal.h"

namespace tlr {

namespace {

constexpr int MC_T = 1024;

// first index of the largest value (ties: smaller index) over the CTA; v >= 0
__device__ void block_argmax(double& v, int& i, double* sv, int* si) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, v, o);
    const int i2 = __shfl_down_sync(0xffffffffu, i, o);
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
  }
  if (lane == 0) { sv[w] = v; si[w] = i; }
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sv[lane] : -1.0;
    i = lane < (int)(blockDim.x >> 5) ? si[lane] : 0x7fffffff;
    for (int o = 16; o; o >>= 1) {
      const double v2 = __shfl_down_sync(0xffffffffu, v, o);
      const int i2 = __shfl_down_sync(0xffffffffu, i, o);
      if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
    if (lane == 0) { sv[0] = v; si[0] = i; }
  }
  __syncthreads();
  v = sv[0];
  i = si[0];
  __syncthreads();
}

// In place: the multipliers of L below the diagonal (unit diagonal; zero at (k+1, k) of a 2x2 block),
// D's diagonal in dd, its subdiagonal in de (nonzero at the first index of a 2x2 block), the block
// sizes in bsz (1 or 2 at a block's first index, 0 at the second), perm[i] = the original index at
// position i.  The interchanges are applied to whole rows (the multipliers left of the step too), so
// that P^T A P = L D L^T with P the accumulated permutation.  Also *delta = sqrt(u / 2) ||A||_inf of
// the input.
__global__ void __launch_bounds__(MC_T) k_bk_ldlt(double* __restrict__ A, int n, int lda, double* __restrict__ dd,
                                                  double* __restrict__ de, int* __restrict__ bsz, int* __restrict__ perm,
                                                  double* __restrict__ delta) {
  extern __shared__ double c0[];  // n: column k before the update; c1: column k + 1 (2x2); w0, w1
  double* c1 = c0 + n;
  double* w0 = c1 + n;
  double* w1 = w0 + n;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_kp, s_step;
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5, nw = T >> 5;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  auto at = [&](int i, int j) -> double& { return A[(size_t)i + (size_t)j * lda]; };  // i >= j
  // ||A||_inf of the symmetric matrix stored in the lower triangle
  double rs = 0.0;
  int ri = 0;
  for (int i = t; i < n; i += T) {
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += fabs(at(i, j));
    for (int j = i + 1; j < n; ++j) s += fabs(at(j, i));
    rs = fmax(rs, s);
  }
  block_argmax(rs, ri, sv, si);
  if (t == 0) *delta = sqrt(2.220446049250313e-16 / 2.0) * rs;
  for (int i = t; i < n; i += T) {
    perm[i] = i;
    bsz[i] = 0;
    de[i] = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n;) {
    // largest entry below the diagonal in column k
    double cm = 0.0;
    int im = 0x7fffffff;
    for (int i = k + 1 + t; i < n; i += T) {
      const double v = fabs(at(i, k));
      if (v > cm || (v == cm && i < im)) { cm = v; im = i; }
    }
    block_argmax(cm, im, sv, si);
    if (t == 0) {
      const double akk = fabs(at(k, k));
      int kp = k, step = 1;
      if (fmax(akk, cm) == 0.0 || akk >= alpha * cm) {
        kp = k;
      } else {
        // largest off-diagonal entry of row / column im of the trailing matrix
        double rm = 0.0;
        for (int j = k; j < im; ++j) rm = fmax(rm, fabs(at(im, j)));
        for (int j = im + 1; j < n; ++j) rm = fmax(rm, fabs(at(j, im)));
        if (akk >= alpha * cm * (cm / rm)) kp = k;
        else if (fabs(at(im, im)) >= alpha * rm) kp = im;
        else { kp = im; step = 2; }
      }
      s_kp = kp;
      s_step = step;
    }
    __syncthreads();
    const int kp = s_kp, step = s_step, kk = k + step - 1;
    if (kp != kk) {  // symmetric interchange of kk and kp (whole rows of the multipliers)
      for (int j = t; j < k; j += T) {
        const double a = at(kk, j);
        at(kk, j) = at(kp, j);
        at(kp, j) = a;
      }
      for (int i = kp + 1 + t; i < n; i += T) {
        const double a = at(i, kk);
        at(i, kk) = at(i, kp);
        at(i, kp) = a;
      }
      for (int j = kk + 1 + t; j < kp; j += T) {
        const double a = at(j, kk);
        at(j, kk) = at(kp, j);
        at(kp, j) = a;
      }
      if (t == 0) {
        const double a = at(kk, kk);
        at(kk, kk) = at(kp, kp);
        at(kp, kp) = a;
        if (step == 2) {
          const double b = at(k + 1, k);
          at(k + 1, k) = at(kp, k);
          at(kp, k) = b;
        }
        const int p = perm[kk];
        perm[kk] = perm[kp];
        perm[kp] = p;
      }
    }
    __syncthreads();
    if (step == 1) {
      const double d = at(k, k);
      for (int i = k + 1 + t; i < n; i += T) c0[i] = at(i, k);
      __syncthreads();
      if (d != 0.0) {
        const double r1 = 1.0 / d;
        for (int j = k + 1 + warp; j < n; j += nw) {  // A22 -= r1 a a^T (lower)
          const double tj = -r1 * c0[j];
          for (int i = j + lane; i < n; i += 32) at(i, j) = fma(c0[i], tj, at(i, j));
        }
        for (int i = k + 1 + t; i < n; i += T) at(i, k) = r1 * c0[i];
      }
      if (t == 0) {
        dd[k] = d;
        bsz[k] = 1;
      }
    } else {
      // 2x2 pivot block D = [a_kk, a_k+1,k; a_k+1,k, a_k+1,k+1]
      const double d21 = at(k + 1, k);
      const double d11 = at(k + 1, k + 1) / d21, d22 = at(k, k) / d21;
      const double tt = 1.0 / (d11 * d22 - 1.0), e21 = tt / d21;
      for (int i = k + 2 + t; i < n; i += T) {
        c0[i] = at(i, k);
        c1[i] = at(i, k + 1);
      }
      __syncthreads();
      for (int j = k + 2 + t; j < n; j += T) {
        w0[j] = e21 * (d11 * c0[j] - c1[j]);
        w1[j] = e21 * (d22 * c1[j] - c0[j]);
      }
      __syncthreads();
      for (int j = k + 2 + warp; j < n; j += nw) {
        const double a0 = w0[j], a1 = w1[j];
        for (int i = j + lane; i < n; i += 32) {
          double a = at(i, j);
          a = fma(-c0[i], a0, a);
          a = fma(-c1[i], a1, a);
          at(i, j) = a;
        }
      }
      for (int j = k + 2 + t; j < n; j += T) {
        at(j, k) = w0[j];
        at(j, k + 1) = w1[j];
      }
      if (t == 0) {
        dd[k] = at(k, k);
        dd[k + 1] = at(k + 1, k + 1);
        de[k] = d21;
        bsz[k] = 2;
        bsz[k + 1] = 0;
      }
    }
    __syncthreads();
    k += step;
  }
}

// raise each pivot block's eigenvalues to at least delta (in place on dd / de)
__device__ void modify_block(double& a, double& c, double& b, double delta) {
  if (c == 0.0) {
    a = fmax(a, delta);
    b = fmax(b, delta);
    return;
  }
  // symmetric Schur decomposition of [a c; c b] (Golub and Van Loan, Algorithm 8.4.1)
  const double tau = (b - a) / (2.0 * c);
  const double tn = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  const double cs = 1.0 / sqrt(1.0 + tn * tn), sn = tn * cs;
  const double l1 = fmax(a - tn * c, delta), l2 = fmax(b + tn * c, delta);
  // [a c; c b] = R diag(l1, l2) R^T with R = [cs sn; -sn cs]
  a = cs * cs * l1 + sn * sn * l2;
  b = sn * sn * l1 + cs * cs * l2;
  c = cs * sn * (l2 - l1);
}

__global__ void k_modify_d(int n, double* dd, double* de, const int* bsz, const double* delta) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double dl = *delta;
  if (bsz[k] == 1) {
    dd[k] = fmax(dd[k], dl);
  } else if (bsz[k] == 2) {
    double a = dd[k], c = de[k], b = dd[k + 1];
    modify_block(a, c, b, dl);
    dd[k] = a;
    de[k] = c;
    dd[k + 1] = b;
  }
}

// L (explicit unit lower, zero at (k+1, k) of a 2x2 block) and W = L (D + F), both n x n (ld n)
__global__ void k_form_lw(int n, const double* __restrict__ F, int lda, const double* __restrict__ dd,
                          const double* __restrict__ de, const int* __restrict__ bsz, double* __restrict__ L,
                          double* __restrict__ W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  auto lij = [&](int r, int c) -> double {
    if (r == c) return 1.0;
    if (r < c) return 0.0;
    if (r == c + 1 && bsz[c] == 2) return 0.0;
    return F[(size_t)r + (size_t)c * lda];
  };
  L[(size_t)i + (size_t)j * n] = lij(i, j);
  double w;
  if (bsz[j] == 1) w = lij(i, j) * dd[j];
  else if (bsz[j] == 2) w = lij(i, j) * dd[j] + lij(i, j + 1) * de[j];
  else w = lij(i, j - 1) * de[j - 1] + lij(i, j) * dd[j];  // second column of a 2x2 block
  W[(size_t)i + (size_t)j * n] = w;
}

// A(perm[i], perm[j]) = (B(i, j) + B(j, i)) / 2 for the tile in its original order
__global__ void k_unpermute_sym(int n, const double* __restrict__ B, const int* __restrict__ perm,
                                double* __restrict__ A, int lda) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const double v = 0.5 * (B[(size_t)i + (size_t)j * n] + B[(size_t)j + (size_t)i * n]);
  A[(size_t)perm[i] + (size_t)perm[j] * lda] = v;
}

}  // namespace

void modified_cholesky_tile(tlr_ctx* ctx, int n, double* A, int lda, double* Linv, int* info, Buf& work,
                            Buf& tmp) {
  if (n <= 0) return;
  const size_t nn = (size_t)n * n;
  double* base = work.need<double>(3 * nn + 3 * (size_t)n + 4);
  double* Lx = base;
  double* W = Lx + nn;
  double* B = W + nn;
  double* dd = B + nn;
  double* de = dd + n;
  double* delta = de + n;
  int* bsz = reinterpret_cast<int*>(delta + 2);
  int* perm = bsz + n + (n & 1);
  TLR_REQUIRE(reinterpret_cast<char*>(perm + n) <= reinterpret_cast<char*>(base + 3 * nn + 3 * (size_t)n + 4),
              TLR_ERR_LIMIT, "modified Cholesky workspace");
  static bool attr = false;
  if (!attr) {
    TLR_CUDA(cudaFuncSetAttribute(k_bk_ldlt, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 2048 * (int)sizeof(double)));
    attr = true;
  }
  TLR_REQUIRE(n <= 2048, TLR_ERR_LIMIT, "modified Cholesky: tile above 2048");
  TLR_SITE_PRE(ctx);
  k_bk_ldlt<<<1, MC_T, 4 * (size_t)n * sizeof(double), ctx->stream>>>(A, n, lda, dd, de, bsz, perm, delta);
  TLR_LAUNCH_CHECK(ctx);
  TLR_SITE_PRE(ctx);
  k_modify_d<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, dd, de, bsz, delta);
  TLR_LAUNCH_CHECK(ctx);
  dim3 g((n + 255) / 256, n);
  TLR_SITE_PRE(ctx);
  k_form_lw<<<g, 256, 0, ctx->stream>>>(n, A, lda, dd, de, bsz, Lx, W);
  TLR_LAUNCH_CHECK(ctx);
  std::vector<GemmJob<double>> jb{job<double>(NT, n, n, W, n, Lx, n, n, B, n, 1.0, 0.0)};
  gemm<double>(ctx, NT, jb);
  TLR_SITE_PRE(ctx);
  k_unpermute_sym<<<g, 256, 0, ctx->stream>>>(n, B, perm, A, lda);
  TLR_LAUNCH_CHECK(ctx);
  // the Cholesky factor of A + E (positive definite up to rounding) and, if asked, its inverse
  TLR_CUDA(cudaMemsetAsync(info, 0xff, sizeof(int), ctx->stream));
  std::vector<DenseTile> t{DenseTile{A, nullptr, info, Linv, n, lda}};
  dense_factor_batch(ctx, t, 0, tmp);
  if (Linv) dense_trinv_batch(ctx, t, 0, tmp);
}

}  // namespace tlr
