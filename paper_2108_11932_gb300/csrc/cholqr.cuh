// Register-resident Cholesky-QR step of the ARA orthogonalization (one warp per slot), shared by the
// stand-alone kernel (k_misc.cu) and the fused orthogonalization round (k_orth.cu).
//
// First pass: G = Y1^T Y1 of the projected panel; the convergence quantity e = sqrt(max_c G_cc) is the
// largest column norm of (I - QQ^T)Y (the a-posteriori test of Algorithm 1).  If e <= thr the slot
// converged and M = 0.  Otherwise an unpivoted Cholesky keeps column j when its pivot (squared norm
// orthogonal to the kept earlier columns) exceeds max(thr^2, tau G_jj); M = E_keep R^{-1} (BS x BS,
// kept columns first, zero columns after), so that W = Y M has orthonormal columns.  Second pass
// (re-orthogonalization): the same on the leading nk x nk block of W^T W with thr = 0.
//
// Lane c holds column c of G.  Right-looking: when column j is kept, every later column c is reduced by
// the rank-one term R(j, :)^T R(j, c); a dropped column leaves the others unchanged.  The kept factor is
// embedded in an upper-triangular Rt whose dropped rows and columns are the identity, so Rt^{-1}
// restricted to the kept indices is the inverse of the kept factor, and every register index is a
// compile-time constant.
#pragma once

namespace tlr {

// G: BS x BS column-major (global or shared); M: BS x BS column-major output; st: the slot's
// {converged, kept} pair; en: the slot's convergence norm (first pass only); nk_in: columns kept by the
// first pass (second pass only).
template <int BS>
__device__ __forceinline__ void cholqr_warp(const double* G, double* M, int* st, double* en, double thr,
                                            double tau, int first_pass, int nk_in) {
  static_assert(BS <= 32, "one lane per column");
  const int lane = threadIdx.x & 31;
  double g[BS];  // column `lane` of G, reduced in place
#pragma unroll
  for (int r = 0; r < BS; ++r) g[r] = (lane < BS) ? G[r + lane * BS] : 0.0;
  double gdiag = 0.0;
#pragma unroll
  for (int r = 0; r < BS; ++r)
    if (r == lane) gdiag = g[r];
  int n = BS;
  double thr2 = thr * thr;
  if (first_pass) {
    double gmax = gdiag;
    for (int o = 16; o; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    const double e = sqrt(fmax(gmax, 0.0));
    if (lane == 0) *en = e;
    if (!(e > thr)) {  // converged (also catches NaN-free zero panels)
      if (lane < BS) {
#pragma unroll
        for (int r = 0; r < BS; ++r) M[r + lane * BS] = 0.0;
      }
      if (lane == 0) { st[0] = 1; st[1] = 0; }
      return;
    }
    if (lane == 0) st[0] = 0;
  } else {
    n = nk_in;
    thr2 = 0.0;
  }
  double rt[BS];      // rt[j] = Rt(j, lane)
  double inv[BS];     // 1 / Rt(j, j), the same in every lane
  unsigned mask = 0;  // kept columns
#pragma unroll
  for (int j = 0; j < BS; ++j) {
    rt[j] = (lane == j) ? 1.0 : 0.0;
    inv[j] = 1.0;
    if (j < n) {
      const double dj = __shfl_sync(0xffffffffu, g[j], j);  // pivot of column j
      const double gjj = __shfl_sync(0xffffffffu, gdiag, j);
      const bool kept = (dj > fmax(thr2, tau * gjj)) && (dj > 0.0) && isfinite(dj);
      if (kept) {
        // every later use multiplies (a warp-wide FP64 divide or square root costs as much as
        // ten FMAs on this part, and the factor and its inverse need 3 BS of them)
        inv[j] = rsqrt(dj);  // one reciprocal square root per pivot; R(j, j) = dj / sqrt(dj)
        const double rjj = dj * inv[j];
        const double rj = (lane == j) ? rjj : ((lane > j && lane < n) ? g[j] * inv[j] : 0.0);
#pragma unroll
        for (int a = j + 1; a < BS; ++a) {
          const double rja = __shfl_sync(0xffffffffu, rj, a);
          if (lane > j && lane < n) g[a] = fma(-rja, rj, g[a]);
        }
        rt[j] = rj;
        mask |= 1u << j;
      }
    }
  }
  // decouple dropped columns: Rt(j, c) = 0 for kept j and dropped c != j
  const bool mine = (lane < BS) && ((mask >> lane) & 1u);
#pragma unroll
  for (int j = 0; j < BS; ++j)
    if (!mine && lane != j) rt[j] = 0.0;
  // column `lane` of Rt^{-1} by back substitution: x[p] = -(sum_{q>p} Rt(p,q) x[q]) / Rt(p,p)
  double x[BS];
#pragma unroll
  for (int p = BS - 1; p >= 0; --p) {
    double acc = 0.0;
#pragma unroll
    for (int q = p + 1; q < BS; ++q) {
      const double rpq = __shfl_sync(0xffffffffu, rt[p], q);
      if (q <= lane) acc = fma(rpq, x[q], acc);
    }
    x[p] = (p == lane) ? inv[p] : ((p < lane) ? -acc * inv[p] : 0.0);
  }
  // M column pos(lane) = kept part of column `lane` of Rt^{-1}; zero elsewhere
  const int nk = __popc(mask);
  if (lane < BS) {
#pragma unroll
    for (int r = 0; r < BS; ++r) M[r + lane * BS] = 0.0;
  }
  __syncwarp();
  if (mine) {
    const int pos = __popc(mask & ((1u << lane) - 1u));
#pragma unroll
    for (int p = 0; p < BS; ++p)
      if (p <= lane && ((mask >> p) & 1u)) M[p + pos * BS] = x[p];
  }
  if (lane == 0) st[1] = nk;
}

}  // namespace tlr
