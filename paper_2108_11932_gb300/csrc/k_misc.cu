// Small and medium kernels of the TLR factorization (everything except the batched GEMM).
#include <math.h>

#include "common.h"
#include "cholqr.cuh"

namespace tlr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------------ Omega (Algorithm 1 randn)
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
// multiplications (0xD2511F53, 0xCD9E8D57) with Weyl key increments
// (0x9E3779B9, 0xBB67AE85).  Counter (pair m, round t, column k, stream),
// key (seed lo, seed hi); Box-Muller turns the 4 words into 2 Gaussians.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__global__ void k_omega(uint32_t s0, uint32_t s1, uint32_t stream, uint32_t k, uint32_t t, int n,
                        double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * m >= n) return;
  uint32_t c[4] = {(uint32_t)m, t, k, stream};
  philox4x32_10(c, s0, s1);
  const uint64_t a = ((uint64_t)c[1] << 32) | c[0];
  const uint64_t w = ((uint64_t)c[3] << 32) | c[2];
  const double u1 = ((double)(a >> 11) + 0.5) * 0x1p-53;
  const double u2 = (double)(w >> 11) * 0x1p-53 + 0x1p-54;
  const double rho = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  out[2 * m] = rho * cs;
  if (2 * m + 1 < n) out[2 * m + 1] = rho * sn;
}

void omega(tlr_ctx* ctx, uint64_t seed, uint32_t stream, uint32_t k, uint32_t t, int b, int bs,
           double* out) {
  const int n = b * bs;
  const int pairs = (n + 1) / 2;
  TLR_SITE_PRE(ctx);
  k_omega<<<cdiv(pairs, 256), 256, 0, ctx->stream>>>((uint32_t)seed, (uint32_t)(seed >> 32), stream,
                                                      k, t, n, out);
  TLR_LAUNCH_CHECK(ctx);
}

// ------------------------------------------------------------------ kernel tiles (Section 6)
// A_ij = exp(-|x_i - x_j| / ell) (+ nugget on the diagonal), evaluated on the integer pipe.  GB300
// retires FP64 at 1/64 of its FP32 rate, so a tile entry computed in FP64 (distance, square root,
// exponential: about 25 FP64 instructions) costs as much as ~800 integer instructions; here an entry
// takes no FP64 instruction at all:
//
//  1. Points on a 64-bit grid (k_grid_points, once per matrix): X = round(x 2^q) - round(o 2^q), o the
//     per-dimension minimum, 2^q the largest power of two with (max - min) 2^q < 2^62.  Differences of
//     grid coordinates are exact, and they equal the FP64 differences whenever the coordinates are
//     multiples of 2^-q (every |x| >= range 2^-9); otherwise they are off by at most 2^-q.
//  2. S = sum_k (X_ik - X_jk)^2 exactly, as a 128-bit integer.
//  3. sqrt(S): normalised to F = S 2^-e in [1, 4), a single-precision rsqrt seed y0 (relative error
//     ~2^-21), then one third-order Newton correction sqrt(F) = F y0 (1 + h/2 + 3h^2/8 + O(h^3)),
//     h = 1 - F y0^2, in 64-bit fixed point (~2^-58 relative).
//  4. z = c sqrt(S) 2^-q with c = 1/ell, then exp(-z) by the table-driven method of Tang (ACM TOMS
//     15(2), 1989) in fixed point: z 64/ln2 = n + f (128-bit product, n = floor, 0 <= f < 1),
//     rho = f ln2/64, exp(-z) = 2^(-n/64) exp(-rho), exp(-rho) by its degree-6 Taylor polynomial in
//     unsigned Horner form (truncation below 2^-58 for rho < ln2/64), 2^(-j/64) from a 64-entry Q63
//     table, then rounded to 53 bits.
//
// Error: under 0.3 x 2^-52 (1 + z) relative (the (1 + z) is the conditioning of exp in its argument,
// which the FP64 formula has as well).  Entries below 2^-1020 (z > 707) are returned as 0.
namespace fx {
// round(64/ln2 2^56), round(ln2/64 2^70), Fk = round(2^62 / k!), TAB[j] = round(2^(63 - j/64))
constexpr uint64_t KQ = 0x5c551d94ae0bf85eull;
constexpr uint64_t L70 = 0xb17217f7d1cf79acull;
constexpr uint64_t F1 = 0x4000000000000000ull, F2 = 0x2000000000000000ull, F3 = 0x0aaaaaaaaaaaaaabull,
                   F4 = 0x02aaaaaaaaaaaaabull, F5 = 0x0088888888888889ull, F6 = 0x0016c16c16c16c17ull;
__device__ const uint64_t TAB[64] = {
    0x8000000000000000ull, 0x7e9f06067a4360baull, 0x7d41d96db915019dull, 0x7be86fb985689ddcull,
    0x7a92be8a92436616ull, 0x7940bb9e2cffd89dull, 0x77f25ccdee6d7ae6ull, 0x76a7980f6cca15c2ull,
    0x75606373ee921c97ull, 0x741cb5281e25ee34ull, 0x72dc8373be41a454ull, 0x719fc4b95f452d29ull,
    0x70666f76154a7089ull, 0x6f307a412f074892ull, 0x6dfddbcbed791babull, 0x6cce8ae13c57ebdbull,
    0x6ba27e656b4eb57aull, 0x6a79ad55e7f6fd10ull, 0x69540ec8f895722dull, 0x683199ed779592caull,
    0x6712460a8fc24072ull, 0x65f60a7f79393e2eull, 0x64dcdec3371793d1ull, 0x63c6ba6455dcd8aeull,
    0x62b39508aa836d6full, 0x61a3666d124bb204ull, 0x6096266533384a2bull, 0x5f8bccdb3d398841ull,
    0x5e8451cfac061b5full, 0x5d7fad59099f22feull, 0x5c7dd7a3b17dcf75ull, 0x5b7ec8f19468bbc9ull,
    0x5a827999fcef3242ull, 0x5988e20954889245ull, 0x5891fac0e95612c8ull, 0x579dbc56b48521baull,
    0x56ac1f752150a563ull, 0x55bd1cdad49f699cull, 0x54d0ad5a753e077cull, 0x53e6c9da74b29ab5ull,
    0x52ff6b54d8a89c75ull, 0x521a8ad704f3404full, 0x513821818624b40cull, 0x50582887dcb8a7e1ull,
    0x4f7a993048d088d7ull, 0x4e9f6cd3967fdba8ull, 0x4dc69cdceaa72a9cull, 0x4cf022c9905bfd32ull,
    0x4c1bf828c6dc54b8ull, 0x4b4a169b900c2d00ull, 0x4a7a77d47f7b84b1ull, 0x49ad159789f37496ull,
    0x48e1e9b9d588e19bull, 0x4818ee218a3358eeull, 0x47521cc5a2e6a9e0ull, 0x468d6fadbf2dd4f3ull,
    0x45cae0f1f545eb73ull, 0x450a6abaa4b77ecdull, 0x444c0740496d4294ull, 0x438fb0cb4f468808ull,
    0x42d561b3e6243d8aull, 0x421d1461d66f2023ull, 0x4166c34c5615d0ecull, 0x40b268f9de0183baull};

// exp(-c sqrt(S) 2^-q) for S = hi 2^64 + lo, c = Cm 2^(ec - 63) (Cm in [2^63, 2^64)), ezb = ec + 63 - q.
__device__ __forceinline__ double entry(uint64_t hi, uint64_t lo, int ezb, uint64_t Cm, const uint64_t* tab) {
  if ((hi | lo) == 0) return 1.0;
  int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  lz &= ~1;  // even shift: sqrt(S) = sqrt(F) 2^(63 - lz/2), F = H / 2^62 in [1, 4)
  uint64_t H;
  if (lz == 0) H = hi;
  else if (lz < 64) H = (hi << lz) | (lo >> (64 - lz));
  else H = lo << (lz - 64);
  const unsigned top = (unsigned)(H >> 63);
  const unsigned fb = ((127u + top) << 23) | (unsigned)((H >> (39 + top)) & 0x7fffffu);
  const unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
  const int ey = (int)((yb >> 23) & 0xffu) - 127;
  const uint64_t Y0 = (uint64_t)((yb & 0x7fffffu) | 0x800000u) << (39 + ey);  // Q62
  const uint64_t G0 = __umul64hi(H, Y0);                                      // F y0, Q60
  const long long h = (long long)((1ull << 58) - __umul64hi(G0, Y0));         // 1 - F y0^2, Q58
  const long long h2 = __mul64hi(h * 32, h * 32);                             // h^2, Q62
  const long long corr = h * 8 + ((3 * h2) >> 3);                             // h/2 + 3h^2/8, Q62
  const uint64_t G = G0 + (uint64_t)(__mul64hi((long long)G0, corr) * 4);     // sqrt(F), Q60
  const uint64_t P = __umul64hi(G, Cm);                                       // z = P 2^(ez - 59)
  const int ez = ezb - lz / 2;
  if (ez >= 10) return 0.0;  // z >= 1024
  const uint64_t phi = __umul64hi(P, KQ), plo = P * KQ;                       // z 64/ln2 = prod 2^(ez - 115)
  const int sh = 115 - ez;
  uint64_t n, frac;                                                           // frac: Q64 fraction of n
  if (sh < 128) {
    n = phi >> (sh - 64);
    frac = (phi << (128 - sh)) | (plo >> (sh - 64));
  } else {
    n = 0;
    frac = sh < 192 ? (phi >> (sh - 128)) : 0;
  }
  if ((n >> 6) > 1020) return 0.0;  // n = floor(z 64/ln2), frac its remainder in [0, 1)
  // exp(-rho) = 1 - rho (F1 - rho (F2 - rho (F3 - rho (F4 - rho (F5 - rho F6))))), all terms >= 0
  const uint64_t rho = __umul64hi(frac, L70);                                 // Q70, in [0, ln2/64)
  uint64_t acc = F5 - (__umul64hi(rho, F6) >> 6);                            // Horner, Q62
  acc = F4 - (__umul64hi(rho, acc) >> 6);
  acc = F3 - (__umul64hi(rho, acc) >> 6);
  acc = F2 - (__umul64hi(rho, acc) >> 6);
  acc = F1 - (__umul64hi(rho, acc) >> 6);
  const uint64_t E = (1ull << 62) - (__umul64hi(rho, acc) >> 6);              // exp(-rho), Q62
  const uint64_t V = __umul64hi(tab[n & 63], E);                              // Q61, in (0.49, 1.01)
  const int lzv = __clzll((long long)V);
  const uint64_t Vn = V << lzv;
  const uint64_t M53 = (Vn >> 11) + ((Vn >> 10) & 1ull);                      // nearest, may carry to 2^53
  const uint64_t bits = ((uint64_t)(1025 - lzv - (int)(n >> 6)) << 52) + (M53 - (1ull << 52));
  return __longlong_as_double((long long)bits);
}
}  // namespace fx

// round(x 2^q) as a 128-bit integer (|x| 2^q < 2^126), halves away from zero.
__device__ __forceinline__ __int128 grid_round(double x, int q) {
  const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bx >> 52) & 0x7ff);
  unsigned long long m = bx & ((1ull << 52) - 1);
  int ex;
  if (E == 0) {
    ex = -1074;
  } else {
    m |= 1ull << 52;
    ex = E - 1075;
  }
  const int sh = ex + q;
  __int128 v;
  if (m == 0) v = 0;
  else if (sh >= 0) v = (__int128)m << sh;
  else if (sh <= -64) v = 0;
  else v = (__int128)(((m >> (-sh - 1)) + 1) >> 1);
  return (bx >> 63) ? -v : v;
}

// Grid scale and offsets of the points (one block): q and o_k = min_k x_k.  Comparisons on
// order-preserving integer images of the FP64 bits.
__device__ __forceinline__ unsigned long long ord_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}
__device__ __forceinline__ double ord_val(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}
__global__ void __launch_bounds__(256) k_grid_range(const double* __restrict__ pts, int64_t N, int d,
                                                    GridInfo* __restrict__ gi) {
  __shared__ unsigned long long smin[3][256], smax[3][256];
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
  for (int64_t p = threadIdx.x; p < N; p += blockDim.x)
    for (int k = 0; k < d; ++k) {
      const unsigned long long key = ord_key(pts[p * d + k]);
      mn[k] = key < mn[k] ? key : mn[k];
      mx[k] = key > mx[k] ? key : mx[k];
    }
  for (int k = 0; k < 3; ++k) { smin[k][threadIdx.x] = mn[k]; smax[k][threadIdx.x] = mx[k]; }
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) {
        const unsigned long long a = smin[k][threadIdx.x + w], c = smax[k][threadIdx.x + w];
        if (a < smin[k][threadIdx.x]) smin[k][threadIdx.x] = a;
        if (c > smax[k][threadIdx.x]) smax[k][threadIdx.x] = c;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double R = 0.0, A = 0.0;
    for (int k = 0; k < d; ++k) {
      const double lo = ord_val(smin[0 + k][0]), hi = ord_val(smax[k][0]);
      gi->o[k] = lo;
      R = fmax(R, hi - lo);
      A = fmax(A, fmax(fabs(lo), fabs(hi)));
    }
    int q = R > 0.0 ? 61 - ilogb(R) : 0;
    if (A > 0.0) q = min(q, 125 - ilogb(A));
    gi->q = q;
  }
}
__global__ void k_grid_points(const double* __restrict__ pts, int64_t n, int d, const GridInfo* __restrict__ gi,
                              long long* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int q = gi->q;
  const int k = (int)(e % d);
  X[e] = (long long)(grid_round(pts[e], q) - grid_round(gi->o[k], q));
}

void grid_points(tlr_ctx* ctx, const double* pts, int64_t N, int d, GridInfo* gi, long long* X) {
  if (N <= 0) return;
  TLR_SITE_PRE(ctx);
  k_grid_range<<<1, 256, 0, ctx->stream>>>(pts, N, d, gi);
  TLR_LAUNCH_CHECK(ctx);
  TLR_SITE_PRE(ctx);
  k_grid_points<<<cdiv(N * d, 256), 256, 0, ctx->stream>>>(pts, N * d, d, gi, X);
  TLR_LAUNCH_CHECK(ctx);
}

// One block per (column group of GT_COLS columns, tile); each thread owns rows tid, tid + 256, ... and
// walks the group's columns, whose grid points sit in shared memory.  With tmax, also records each
// tile's largest entry (as FP64 bits: the entries are >= 0, so the bit patterns order like the values;
// zeroed by the caller).
constexpr int GT_COLS = 16, GT_THREADS = 256;
template <int D>
__global__ void __launch_bounds__(GT_THREADS) k_gen_tiles(const long long* __restrict__ X,
                                                          const GridInfo* __restrict__ gi, int64_t N, uint64_t Cm,
                                                          int ec, double one_nug, int b, const int* __restrict__ ij,
                                                          double* __restrict__ out,
                                                          unsigned long long* __restrict__ tmax) {
  __shared__ uint64_t tab[64];
  __shared__ long long xc[GT_COLS * D];
  const int t = blockIdx.y;
  const int i = ij[2 * t], j = ij[2 * t + 1];
  const int c0 = blockIdx.x * GT_COLS, nc = min(GT_COLS, b - c0);
  if (threadIdx.x < 64) tab[threadIdx.x] = fx::TAB[threadIdx.x];
  if (threadIdx.x < nc * D) {
    const int64_t gj = (int64_t)j * b + c0 + threadIdx.x / D;
    xc[threadIdx.x] = gj < N ? X[gj * D + threadIdx.x % D] : 0;
  }
  __syncthreads();
  const int ezb = ec + 63 - gi->q;
  double* T = out + (size_t)t * b * b + (size_t)c0 * b;
  unsigned long long vmax = 0;
  for (int r = threadIdx.x; r < b; r += GT_THREADS) {
    const int64_t g_i = (int64_t)i * b + r;
    long long xr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xr[k] = g_i < N ? X[g_i * D + k] : 0;
    for (int c = 0; c < nc; ++c) {
      const int64_t g_j = (int64_t)j * b + c0 + c;
      double v;
      if (g_i < N && g_j < N) {
        uint64_t hi = 0, lo = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const long long df = xr[k] - xc[c * D + k];
          const uint64_t a = (uint64_t)(df < 0 ? -df : df);
          const uint64_t l = a * a;
          lo += l;
          hi += __umul64hi(a, a) + (lo < l ? 1ull : 0ull);
        }
        v = g_i == g_j ? one_nug : fx::entry(hi, lo, ezb, Cm, tab);  // exp(0) + nugget on the diagonal
      } else {
        v = (g_i == g_j) ? 1.0 : 0.0;  // identity padding of a ragged last tile
      }
      T[r + (size_t)c * b] = v;
      const unsigned long long vb = (unsigned long long)__double_as_longlong(v);
      vmax = vb > vmax ? vb : vmax;
    }
  }
  if (tmax) {
    for (int o = 16; o; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, vmax, o);
      vmax = w > vmax ? w : vmax;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(tmax + t, vmax);
  }
}

void gen_tiles(tlr_ctx* ctx, const long long* X, const GridInfo* gi, int64_t N, int d, double ell, double nugget,
               int b, const int* tile_ij, int ntiles, double* out, unsigned long long* tmax) {
  if (ntiles <= 0) return;
  TLR_REQUIRE(d >= 1 && d <= 3, TLR_ERR_ARG, "points of dimension 1 to 3");
  int ec = 0;
  const double mc = frexp(1.0 / ell, &ec);  // 1/ell = mc 2^ec, mc in [1/2, 1)
  const uint64_t Cm = (uint64_t)ldexp(mc, 64);
  ec -= 1;
  dim3 grid(cdiv(b, GT_COLS), (unsigned)ntiles);
  TLR_SITE_PRE(ctx);
  if (d == 1)
    k_gen_tiles<1><<<grid, GT_THREADS, 0, ctx->stream>>>(X, gi, N, Cm, ec, 1.0 + nugget, b, tile_ij, out, tmax);
  else if (d == 2)
    k_gen_tiles<2><<<grid, GT_THREADS, 0, ctx->stream>>>(X, gi, N, Cm, ec, 1.0 + nugget, b, tile_ij, out, tmax);
  else
    k_gen_tiles<3><<<grid, GT_THREADS, 0, ctx->stream>>>(X, gi, N, Cm, ec, 1.0 + nugget, b, tile_ij, out, tmax);
  TLR_LAUNCH_CHECK(ctx);
}

// ------------------------------------------------------------------ Cholesky-QR with dropping
// One warp per slot.  First pass: G = Y1^T Y1 of the projected panel; the
// convergence quantity e = sqrt(max_c G_cc) = max column norm of (I - QQ^T)Y.
// If e <= thr the slot converged and M = 0.  Otherwise an unpivoted Cholesky
// keeps column j when its pivot (squared norm orthogonal to the kept earlier
// columns) exceeds max(thr^2, tau * G_jj); M = E_keep R^{-1} (bs x bs, kept
// columns first, zero columns after), so W = Y M has orthonormal-ish columns.
// Second pass (re-orthogonalization): same on the leading nk x nk block of
// W^T W with thr = 0.
constexpr int MAXBS = 64;
__global__ void __launch_bounds__(32) k_cholqr_small(int bs, const double* __restrict__ Gall,
                                                     double* __restrict__ Mall, int* __restrict__ status,
                                                     double* __restrict__ enorm, const double* __restrict__ thrv,
                                                     double tau, int first_pass, const int* __restrict__ nk_in) {
  extern __shared__ double dsm[];
  const int ld = bs + 1;
  double* Rm = dsm;                 // bs x (bs + 1), row-major R(row, col)
  double* Rim = dsm + bs * ld;      // inverse of the kept factor
  int* keep = reinterpret_cast<int*>(dsm + 2 * bs * ld);
#define R(r, c) Rm[(r) * ld + (c)]
#define Ri(r, c) Rim[(r) * ld + (c)]
  const int s = blockIdx.x, lane = threadIdx.x;
  const double* G = Gall + (size_t)s * bs * bs;
  double* M = Mall + (size_t)s * bs * bs;
  for (int e = lane; e < bs * bs; e += 32) M[e] = 0.0;
  int n = bs;
  const double thr = thrv[s];
  double thr2 = thr * thr;
  if (first_pass) {
    double gmax = 0.0;
    for (int c = lane; c < bs; c += 32) gmax = fmax(gmax, G[c + (size_t)c * bs]);
    for (int o = 16; o; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    const double e = sqrt(fmax(gmax, 0.0));
    if (lane == 0) enorm[s] = e;
    if (!(e > thr)) {  // converged (also catches NaN-free zero panels)
      if (lane == 0) { status[2 * s] = 1; status[2 * s + 1] = 0; }
      return;
    }
    if (lane == 0) status[2 * s] = 0;
  } else {
    n = nk_in[2 * s + 1];
    thr2 = 0.0;
    if (n <= 0) {
      if (lane == 0) status[2 * s + 1] = 0;
      return;
    }
  }
  int nk = 0;
  for (int j = 0; j < n; ++j) {
    // R(keep[p], j) for kept rows, in order
    for (int p = 0; p < nk; ++p) {
      const int l = keep[p];
      double part = 0.0;
      for (int q = lane; q < p; q += 32) part = fma(R(keep[q], l), R(keep[q], j), part);
      for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) R(l, j) = (G[l + (size_t)j * bs] - part) / R(l, l);
      __syncwarp();
    }
    double part = 0.0;
    for (int q = lane; q < nk; q += 32) part = fma(R(keep[q], j), R(keep[q], j), part);
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const double gjj = G[j + (size_t)j * bs];
    const double dpiv = gjj - part;
    const bool kept = (dpiv > fmax(thr2, tau * gjj)) && (dpiv > 0.0) && isfinite(dpiv);
    if (kept) {
      if (lane == 0) { R(j, j) = sqrt(dpiv); keep[nk] = j; }
      ++nk;
    }
    __syncwarp();
  }
  // Rinv = inverse of the kept upper-triangular factor (nk x nk), column per lane.
  for (int c = lane; c < nk; c += 32) {
    Ri(c, c) = 1.0 / R(keep[c], keep[c]);
    for (int p = c - 1; p >= 0; --p) {
      double acc = 0.0;
      for (int q = p + 1; q <= c; ++q) acc = fma(R(keep[p], keep[q]), Ri(q, c), acc);
      Ri(p, c) = -acc / R(keep[p], keep[p]);
    }
  }
  __syncwarp();
  for (int e = lane; e < nk * nk; e += 32) {
    const int p = e % nk, c = e / nk;
    if (p <= c) M[keep[p] + (size_t)c * bs] = Ri(p, c);
  }
  if (lane == 0) status[2 * s + 1] = nk;
#undef R
#undef Ri
}

// Register-resident Cholesky-QR step for bs <= 32 (one warp per slot, lane c holds column c of the
// Gram matrix): the same decisions as k_cholqr_small, computed right-looking (cholqr.cuh).
template <int BS>
__global__ void __launch_bounds__(32) k_cholqr_reg(const double* __restrict__ Gall, double* __restrict__ Mall,
                                                   int* __restrict__ status, double* __restrict__ enorm,
                                                   const double* __restrict__ thrv, double tau, int first_pass,
                                                   const int* __restrict__ nk_in) {
  const int s = blockIdx.x;
  cholqr_warp<BS>(Gall + (size_t)s * BS * BS, Mall + (size_t)s * BS * BS, status + 2 * s, enorm + s, thrv[s], tau,
                  first_pass, first_pass ? 0 : nk_in[2 * s + 1]);
}

void cholqr_small(tlr_ctx* ctx, int nslots, int bs, const double* G, double* Mout, int* status,
                  double* enorm, const double* thr, double tau, int first_pass, const int* nk_in) {
  if (nslots <= 0) return;
  if (bs == 16 || bs == 32 || bs == 8) {
    TLR_SITE_PRE(ctx);
    if (bs == 16)
      k_cholqr_reg<16><<<(unsigned)nslots, 32, 0, ctx->stream>>>(G, Mout, status, enorm, thr, tau, first_pass, nk_in);
    else if (bs == 32)
      k_cholqr_reg<32><<<(unsigned)nslots, 32, 0, ctx->stream>>>(G, Mout, status, enorm, thr, tau, first_pass, nk_in);
    else
      k_cholqr_reg<8><<<(unsigned)nslots, 32, 0, ctx->stream>>>(G, Mout, status, enorm, thr, tau, first_pass, nk_in);
    TLR_LAUNCH_CHECK(ctx);
    return;
  }
  TLR_REQUIRE(bs <= MAXBS, TLR_ERR_LIMIT, "ARA block width above 64");
  const size_t smem = sizeof(double) * 2 * bs * (bs + 1) + sizeof(int) * bs;
  static bool attr_set = false;
  if (!attr_set) {
    TLR_CUDA(cudaFuncSetAttribute(k_cholqr_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * 2 * MAXBS * (MAXBS + 1) + sizeof(int) * MAXBS)));
    attr_set = true;
  }
  TLR_SITE_PRE(ctx);
  k_cholqr_small<<<(unsigned)nslots, 32, smem, ctx->stream>>>(bs, G, Mout, status, enorm, thr, tau,
                                                               first_pass, nk_in);
  TLR_LAUNCH_CHECK(ctx);
}

// ------------------------------------------------------------------ dense diagonal-tile factorization
// All kernels take an array of per-tile descriptors (grid.y = tile), so the
// diagonal tiles of many matrices factor in the same launches.
//
// GB300 retires about one warp-wide FP64 FMA per SMSP every 64 clocks, so these
// kernels are built around two rules: keep the sequential pivot chain short (one
// barrier and one reciprocal per column) and spread the FMAs of each step evenly
// over all threads of the CTA.
//
// k_potrf_inv_block: factor the nbk x nbk diagonal block at A (lda) in shared
// memory and write the inverse of its factor to Binv (lower, zeros above the
// diagonal), one CTA of 256 threads per block.
//   Factorization: right-looking elimination on the unscaled columns,
//   a_rc -= a_rj a_cj / a_jj for j < c <= r, which is the Schur-complement step of
//   both Cholesky and unpivoted LDL^T (Section 5.3); afterwards Cholesky takes
//   l_jj = sqrt(a_jj), l_rj = a_rj / l_jj and LDL^T takes d_j = a_jj, l_rj = a_rj / d_j
//   with a unit diagonal.  The trailing triangle of column j is enumerated through
//   a table of (r, c) pairs ordered by descending column, so that it is a prefix of
//   the table and 256 threads share it evenly; thread 0 updates the next pivot
//   first and takes its reciprocal while the others finish the step.
//   Inverse: X = L^{-1} by row elimination; step r subtracts l_r'r X[r, :] from
//   every later row r' and the last update of a row applies its 1 / l_rr.
// A pivot that is not positive (Cholesky) or is zero / not finite (LDL^T) records
// the first failing column in *info (atomicCAS from -1) and stops the block.
constexpr int PB = 64;
static size_t potrf_inv_smem() { return sizeof(double) * 2 * PB * (PB + 1); }

__global__ void __launch_bounds__(256) k_potrf_inv_block(const PotrfJob* __restrict__ jobs, int ldl) {
  const PotrfJob J = jobs[blockIdx.y];
  const int nbk = J.nbk, lda = J.lda;
  double* A = J.A;
  extern __shared__ double dsm[];
  double (*S)[PB + 1] = reinterpret_cast<double (*)[PB + 1]>(dsm);
  double (*X)[PB + 1] = reinterpret_cast<double (*)[PB + 1]>(dsm + PB * (PB + 1));
  __shared__ double ip[PB];   // 1 / a_jj
  __shared__ double idg[PB];  // 1 / l_jj (1 for LDL^T)
  __shared__ unsigned short tab[PB * (PB + 1) / 2];
  __shared__ int fail;
  const int tid = threadIdx.x;
  for (int e = tid; e < nbk * nbk; e += blockDim.x) {
    const int r = e % nbk, c = e / nbk;
    S[r][c] = (r >= c) ? A[r + (size_t)c * lda] : 0.0;
  }
  if (tid < nbk) {  // column c = nbk-1-t occupies entries [t(t+1)/2, t(t+1)/2 + t]
    const int c = nbk - 1 - tid, s0 = tid * (tid + 1) / 2;
    for (int r = c; r < nbk; ++r) tab[s0 + r - c] = (unsigned short)(r | (c << 8));
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  auto bad = [&](double v) { return ldl ? (v == 0.0 || !isfinite(v)) : (!(v > 0.0) || !isfinite(v)); };
  if (tid == 0) {
    const double v = S[0][0];
    if (bad(v)) { fail = 1; atomicCAS(J.info, -1, J.col0); }
    else ip[0] = 1.0 / v;
  }
  __syncthreads();
  for (int j = 0; j + 1 < nbk; ++j) {
    if (fail) break;
    const int m = nbk - 1 - j, Tj = m * (m + 1) / 2, skip = Tj - m;  // skip: entry of (j+1, j+1)
    const double ipj = ip[j];
    if (tid == 0) {
      const double v = fma(-S[j + 1][j], S[j + 1][j] * ipj, S[j + 1][j + 1]);
      S[j + 1][j + 1] = v;
      if (bad(v)) { fail = 1; atomicCAS(J.info, -1, J.col0 + j + 1); }
      else ip[j + 1] = 1.0 / v;
    }
    for (int e = tid; e < Tj; e += blockDim.x) {
      if (e == skip) continue;
      const int rc = tab[e], r = rc & 255, c = rc >> 8;
      S[r][c] = fma(-S[r][j], S[c][j] * ipj, S[r][c]);
    }
    __syncthreads();
  }
  if (fail) return;
  // scale the columns: L in S, 1 / l_jj in idg
  if (tid < nbk) idg[tid] = ldl ? 1.0 : 1.0 / sqrt(S[tid][tid]);
  __syncthreads();
  for (int e = tid; e < nbk * nbk; e += blockDim.x) {
    const int r = e % nbk, c = e / nbk;
    double x = 0.0;
    if (r > c) S[r][c] = S[r][c] * (ldl ? ip[c] : idg[c]);
    if (r == c) x = idg[r];
    X[r][c] = x;
  }
  __syncthreads();
  if (tid < nbk) {
    if (ldl) { J.dvec[J.col0 + tid] = S[tid][tid]; S[tid][tid] = 1.0; }
    else S[tid][tid] = sqrt(S[tid][tid]);
  }
  __syncthreads();
  // X = L^{-1}: step r reads the finished row r and updates rows r' > r, columns c <= r
  for (int r = 0; r + 1 < nbk; ++r) {
    const int w = r + 1, cnt = (nbk - 1 - r) * w;
    for (int e = tid; e < cnt; e += blockDim.x) {
      const int rr = r + 1 + e / w, c = e % w;
      double v = fma(-S[rr][r], X[r][c], X[rr][c]);
      if (rr == r + 1) v *= idg[rr];
      X[rr][c] = v;
    }
    __syncthreads();
  }
  for (int e = tid; e < nbk * nbk; e += blockDim.x) {
    const int r = e % nbk, c = e / nbk;
    if (r >= c) A[r + (size_t)c * lda] = S[r][c];
    J.Binv[r + (size_t)c * J.ldb] = (r >= c) ? X[r][c] : 0.0;
  }
}

// Panel below a factored block, in place: X (m x nbk) <- X Binv^T (Cholesky:
// X L^{-T}), or for LDL^T W <- X Binv^T and X <- W D^{-1}.  Each CTA owns 8 whole
// rows, so it reads them completely before writing them back; thread (r, g) forms
// columns g, g + 16, g + 32, g + 48 of row r, which balances the triangular
// reductions across warps.
__global__ void __launch_bounds__(128) k_panel_apply(const PanelJob* __restrict__ jobs, int ldl) {
  const PanelJob J = jobs[blockIdx.y];
  const int nbk = J.nbk, m = J.m;
  const int tid = threadIdx.x, r0 = blockIdx.x * 8;
  if (r0 >= m) return;
  __shared__ double Bs[PB][PB + 1];
  __shared__ double Xs[8][PB + 1];
  for (int e = tid; e < nbk * nbk; e += 128) {
    const int r = e % nbk, c = e / nbk;
    Bs[r][c] = J.Binv[r + (size_t)c * J.ldb];
  }
  const int rows = min(8, m - r0);
  for (int e = tid; e < 8 * nbk; e += 128) {
    const int r = e % 8, c = e / 8;
    Xs[r][c] = r < rows ? J.X[(r0 + r) + (size_t)c * J.ldx] : 0.0;
  }
  __syncthreads();
  const int r = tid & 7, g = tid >> 3;
  double out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = g + 16 * q;
    double v = 0.0;
    if (c < nbk)
      for (int l = 0; l <= c; ++l) v = fma(Xs[r][l], Bs[c][l], v);
    out[q] = v;
  }
  if (r >= rows) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = g + 16 * q;
    if (c >= nbk) continue;
    const size_t gi = (r0 + r) + (size_t)c * J.ldx;
    if (ldl) {
      J.W[(r0 + r) + (size_t)c * m] = out[q];
      J.X[gi] = out[q] / J.dvec[c];
    } else {
      J.X[gi] = out[q];
    }
  }
}

static size_t two_block_smem() { return sizeof(double) * 2 * PB * (PB + 1); }

// X (nbk x nrhs) <- L^{-1} X (or L^{-T} X if trans), L the nbk x nbk lower
// diagonal block (unit if `unit`).  One thread per right-hand-side column; 64
// columns per CTA.
__global__ void __launch_bounds__(64) k_trsm_left_block(const LeftJob* __restrict__ jobs, int unit, int trans) {
  const LeftJob J = jobs[blockIdx.y];
  const int nbk = J.nbk, nrhs = J.nrhs;
  const int tid = threadIdx.x, c0 = blockIdx.x * PB;
  if (c0 >= nrhs) return;
  extern __shared__ double dsm[];
  double (*Ls)[PB + 1] = reinterpret_cast<double (*)[PB + 1]>(dsm);
  double (*Xs)[PB + 1] = reinterpret_cast<double (*)[PB + 1]>(dsm + PB * (PB + 1));
  for (int e = tid; e < nbk * nbk; e += 64) {
    const int r = e % nbk, c = e / nbk;
    Ls[r][c] = J.L[r + (size_t)c * J.lda];
  }
  const int cols = min(PB, nrhs - c0);
  for (int e = tid; e < nbk * cols; e += 64) {
    const int r = e % nbk, c = e / nbk;
    Xs[r][c] = J.X[r + (size_t)(c0 + c) * J.ldx];
  }
  __syncthreads();
  if (tid < cols) {
    if (!trans) {
      for (int r = 0; r < nbk; ++r) {
        double v = Xs[r][tid];
        for (int l = 0; l < r; ++l) v = fma(-Ls[r][l], Xs[l][tid], v);
        Xs[r][tid] = unit ? v : v / Ls[r][r];
      }
    } else {  // L^T x = b: backward substitution
      for (int r = nbk - 1; r >= 0; --r) {
        double v = Xs[r][tid];
        for (int l = r + 1; l < nbk; ++l) v = fma(-Ls[l][r], Xs[l][tid], v);
        Xs[r][tid] = unit ? v : v / Ls[r][r];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < nbk * cols; e += 64) {
    const int r = e % nbk, c = e / nbk;
    J.X[r + (size_t)(c0 + c) * J.ldx] = Xs[r][c];
  }
}

static void smem_attrs() {
  static bool done = false;
  if (done) return;
  TLR_CUDA(cudaFuncSetAttribute(k_potrf_inv_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_inv_smem()));
  TLR_CUDA(cudaFuncSetAttribute(k_trsm_left_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)two_block_smem()));
  done = true;
}

void potrf_inv_blocks(tlr_ctx* ctx, std::vector<PotrfJob>& jobs, int ldl) {
  smem_attrs();
  for (size_t o = 0; o < jobs.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, jobs.size() - o);
    TLR_REQUIRE(std::all_of(jobs.begin() + o, jobs.begin() + o + cnt, [](const PotrfJob& j) { return j.nbk <= PB; }),
                TLR_ERR_LIMIT, "potrf block above 64");
    const PotrfJob* dj = static_cast<const PotrfJob*>(upload(ctx, jobs.data() + o, cnt * sizeof(PotrfJob)));
    TLR_SITE_PRE(ctx);
    k_potrf_inv_block<<<dim3(1, (unsigned)cnt), 256, potrf_inv_smem(), ctx->stream>>>(dj, ldl);
    TLR_LAUNCH_CHECK(ctx);
  }
}
void panel_apply(tlr_ctx* ctx, std::vector<PanelJob>& jobs, int ldl) {
  int mx = 0;
  std::vector<PanelJob> nz;
  for (auto& j : jobs)
    if (j.m > 0) { nz.push_back(j); mx = std::max(mx, j.m); }
  for (size_t o = 0; o < nz.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, nz.size() - o);
    const PanelJob* dj = static_cast<const PanelJob*>(upload(ctx, nz.data() + o, cnt * sizeof(PanelJob)));
    TLR_SITE_PRE(ctx);
    k_panel_apply<<<dim3(cdiv(mx, 8), (unsigned)cnt), 128, 0, ctx->stream>>>(dj, ldl);
    TLR_LAUNCH_CHECK(ctx);
  }
}
void trsm_lefts(tlr_ctx* ctx, std::vector<LeftJob>& jobs, int unit, int trans) {
  smem_attrs();
  int mx = 0;
  std::vector<LeftJob> nz;
  for (auto& j : jobs)
    if (j.nrhs > 0) { nz.push_back(j); mx = std::max(mx, j.nrhs); }
  for (size_t o = 0; o < nz.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, nz.size() - o);
    const LeftJob* dj = static_cast<const LeftJob*>(upload(ctx, nz.data() + o, cnt * sizeof(LeftJob)));
    TLR_SITE_PRE(ctx);
    k_trsm_left_block<<<dim3(cdiv(mx, PB), (unsigned)cnt), 64, two_block_smem(), ctx->stream>>>(dj, unit, trans);
    TLR_LAUNCH_CHECK(ctx);
  }
}

void trsm_left_block(tlr_ctx* ctx, int nbk, const double* L, int lda, int unit, int nrhs, double* X, int ldx) {
  std::vector<LeftJob> j{LeftJob{L, X, lda, ldx, nrhs, nbk}};
  trsm_lefts(ctx, j, unit, 0);
}
void trsm_left_t_block(tlr_ctx* ctx, int nbk, const double* L, int lda, int unit, int nrhs, double* X, int ldx) {
  std::vector<LeftJob> j{LeftJob{L, X, lda, ldx, nrhs, nbk}};
  trsm_lefts(ctx, j, unit, 1);
}

// ------------------------------------------------------------------ elementwise helpers
__global__ void k_scale_rows(int m, int n, const double* __restrict__ dv, int inv, const double* X,
                             int ldx, double* Y, int ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    const double s = inv ? 1.0 / dv[r] : dv[r];
    Y[r + (size_t)c * ldy] = X[r + (size_t)c * ldx] * s;
  }
}
void scale_rows(tlr_ctx* ctx, int m, int n, const double* dvec, int inv, const double* X, int ldx,
                double* Y, int ldy) {
  if ((int64_t)m * n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_scale_rows<<<std::min<unsigned>(cdiv((int64_t)m * n, 256), 4096u), 256, 0, ctx->stream>>>(
      m, n, dvec, inv, X, ldx, Y, ldy);
  TLR_LAUNCH_CHECK(ctx);
}

__global__ void k_add_diag(int n, double* A, int lda, double s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + (size_t)i * lda] += s;
}
void add_diag(tlr_ctx* ctx, int n, double* A, int lda, double s) {
  TLR_SITE_PRE(ctx);
  k_add_diag<<<cdiv(n, 256), 256, 0, ctx->stream>>>(n, A, lda, s);
  TLR_LAUNCH_CHECK(ctx);
}

// A_ii += sum_j |E_ij| (diagonal compensation, Section 5.1.1); one warp per row.
__global__ void k_add_rowsum_abs(int n, const double* __restrict__ E, int lde, double* A, int lda) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += fabs(E[row + (size_t)c * lde]);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) A[row + (size_t)row * lda] += s;
}
void add_rowsum_abs(tlr_ctx* ctx, int n, const double* E, int lde, double* A, int lda) {
  TLR_SITE_PRE(ctx);
  k_add_rowsum_abs<<<cdiv(n, 8), 256, 0, ctx->stream>>>(n, E, lde, A, lda);
  TLR_LAUNCH_CHECK(ctx);
}

// Deterministic log|det| reduction over the diagonals (fixed thread-to-entry map).
__global__ void __launch_bounds__(1024) k_logdet(int n, const double* __restrict__ diag, int b,
                                                 const double* __restrict__ dvec, double* out) {
  __shared__ double ssum[32];
  __shared__ int sneg[32];
  double s = 0.0;
  int neg = 0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    double v;
    if (dvec) v = dvec[g];
    else {
      const int k = g / b, r = g % b;
      v = diag[(size_t)k * b * b + r + (size_t)r * b];
    }
    s += log(fabs(v));
    neg += (v < 0.0);
  }
  for (int o = 16; o; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    neg += __shfl_xor_sync(0xffffffffu, neg, o);
  }
  if ((threadIdx.x & 31) == 0) { ssum[threadIdx.x / 32] = s; sneg[threadIdx.x / 32] = neg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    int ng = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) { t += ssum[w]; ng += sneg[w]; }
    out[0] = dvec ? t : 2.0 * t;
    out[1] = (double)ng;
  }
}
void logdet_reduce(tlr_ctx* ctx, int n, const double* diag_tiles, int b, int nb, const double* dvec,
                   double* out2) {
  (void)nb;
  TLR_SITE_PRE(ctx);
  k_logdet<<<1, 1024, 0, ctx->stream>>>(n, diag_tiles, b, dvec, out2);
  TLR_LAUNCH_CHECK(ctx);
}

// Exact kernel product Y = A X, A_ij = exp(-|x_i - x_j| / ell) + nugget delta_ij,
// one thread per row, points of the column block staged in shared memory.
constexpr int KMV_T = 128, KMV_R = 8;
__global__ void __launch_bounds__(KMV_T) k_kernel_matvec(const double* __restrict__ pts, int64_t N, int d,
                                                        double inv_ell, double nugget, int nr,
                                                        const double* __restrict__ X, int64_t ldx,
                                                        double* __restrict__ Y, int64_t ldy) {
  __shared__ double P[KMV_T][3];
  __shared__ double Xs[KMV_T][KMV_R];
  const int64_t i = blockIdx.x * (int64_t)KMV_T + threadIdx.x;
  double xi[3] = {0, 0, 0};
  if (i < N)
    for (int q = 0; q < d; ++q) xi[q] = pts[i * d + q];
  double acc[KMV_R] = {0, 0, 0, 0};
  for (int64_t j0 = 0; j0 < N; j0 += KMV_T) {
    const int64_t j = j0 + threadIdx.x;
    __syncthreads();
    if (j < N) {
      for (int q = 0; q < d; ++q) P[threadIdx.x][q] = pts[j * d + q];
      for (int c = 0; c < nr; ++c) Xs[threadIdx.x][c] = X[j + c * ldx];
    }
    __syncthreads();
    const int cnt = (N - j0 < KMV_T) ? (int)(N - j0) : KMV_T;
    for (int jj = 0; jj < cnt; ++jj) {
      double s = 0.0;
      for (int q = 0; q < d; ++q) {
        const double df = xi[q] - P[jj][q];
        s = fma(df, df, s);
      }
      const double a = exp(-sqrt(s) * inv_ell);
      for (int c = 0; c < nr; ++c) acc[c] = fma(a, Xs[jj][c], acc[c]);
    }
  }
  if (i < N)
    for (int c = 0; c < nr; ++c) Y[i + c * ldy] = acc[c] + nugget * X[i + c * ldx];
}
void kernel_matvec(tlr_ctx* ctx, const double* pts, int64_t N, int d, double ell, double nugget,
                   int nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  for (int c0 = 0; c0 < nrhs; c0 += KMV_R) {
    const int nr = std::min(KMV_R, nrhs - c0);
    TLR_SITE_PRE(ctx);
    k_kernel_matvec<<<cdiv(N, KMV_T), KMV_T, 0, ctx->stream>>>(pts, N, d, 1.0 / ell, nugget, nr,
                                                              X + c0 * ldx, ldx, Y + c0 * ldy, ldy);
    TLR_LAUNCH_CHECK(ctx);
  }
}

// Row permutation between the original order and the KD (padded) order.
// gather: Y[p] = X[idx[p]] for p < n_out (rows n_out..n_pad-1 of Y zeroed);
// scatter: Y[idx[p]] = X[p] for p < n_out.
__global__ void k_permute(int64_t n_out, int nrhs, const int64_t* __restrict__ idx, int gather,
                          const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy,
                          int64_t n_pad) {
  const int64_t tot = (gather ? n_pad : n_out) * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rows = gather ? n_pad : n_out;
    const int64_t p = e % rows;
    const int c = (int)(e / rows);
    if (gather) Y[p + c * ldy] = (p < n_out) ? X[idx[p] + c * ldx] : 0.0;
    else Y[idx[p] + c * ldy] = X[p + c * ldx];
  }
}
void permute_rows(tlr_ctx* ctx, int64_t n_out, int nrhs, const int64_t* idx, int gather,
                  const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t n_pad) {
  const int64_t tot = (gather ? n_pad : n_out) * nrhs;
  if (tot <= 0) return;
  TLR_SITE_PRE(ctx);
  k_permute<<<std::min<unsigned>(cdiv(tot, 256), 8192u), 256, 0, ctx->stream>>>(n_out, nrhs, idx, gather,
                                                                               X, ldx, Y, ldy, n_pad);
  TLR_LAUNCH_CHECK(ctx);
}

__global__ void k_copy_matrix(int m, int n, const double* __restrict__ X, int ldx, double* __restrict__ Y,
                              int ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    Y[r + (size_t)c * ldy] = X[r + (size_t)c * ldx];
  }
}
void copy_matrix(tlr_ctx* ctx, int m, int n, const double* X, int ldx, double* Y, int ldy) {
  if ((int64_t)m * n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_copy_matrix<<<std::min<unsigned>(cdiv((int64_t)m * n, 256), 8192u), 256, 0, ctx->stream>>>(m, n, X, ldx,
                                                                                              Y, ldy);
  TLR_LAUNCH_CHECK(ctx);
}

__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}
__global__ void k_to_double(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
}
void to_float(tlr_ctx* ctx, int64_t n, const double* x, float* y) {
  if (n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_to_float<<<std::min<unsigned>(cdiv(n, 256), 8192u), 256, 0, ctx->stream>>>(n, x, y);
  TLR_LAUNCH_CHECK(ctx);
}
void to_double(tlr_ctx* ctx, int64_t n, const float* x, double* y) {
  if (n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_to_double<<<std::min<unsigned>(cdiv(n, 256), 8192u), 256, 0, ctx->stream>>>(n, x, y);
  TLR_LAUNCH_CHECK(ctx);
}

// ------------------------------------------------------------------ block-diagonal Gram products
// Sampling chain with the Gram factor G_ij = V_ij^T [D_j] V_kj (Equation 2 /
// Equation 3 regrouped): the sample of tile i is
//   Y_i = U0_ik (V0_ik^T Omega) - sum_j U_ij (G_ij (U_kj^T Omega))
//       = [U0_ik | U_i0 ... U_i,k-1] W_i,
//   W_i = [X0_i ; -G_i0 X_0 ; ... ; -G_i,k-1 X_k-1],  X_j = U_kj^T Omega, X0_i = V0_ik^T Omega.
// G for block column j is stored as Gcol_j = V(j)[tiles i >= k]^T [D_j] V_kj
// (rows grouped by i at V's column offsets, leading dimension gld[j]).
// Every slot carries its own matrix's tables, so slots of different matrices share
// one launch.  Grid (slot, j in 0..kmax): block j < k writes -G_ij X_j, block k copies X0_i.
//
// The projection (sampleLeftT) uses the same blocks transposed:
//   B_i = T_ik^T Q_i = [V0_ik | U_k0 ... U_k,k-1] Z_i with
//   P_i = [U0_ik | U_i0 ...]^T Q_i ((r0 + K_i) x q),
//   Z_i = [P_i^(0) ; -G_i0^T P_i^(j=0 block) ; ...]   ((r0 + K_k) x q).
//
// Work is split into 16 x 16 output tiles: item (slot, j, row chunk, column chunk)
// computes out = -op(G_ij) In on its tile over the whole inner dimension K, with
// 16-deep chunks of both operands staged in shared memory and two accumulators per
// thread.  Large blocks (ranks near the diagonal reach 10x the mean) are spread
// over many CTAs instead of serializing on one SM's FP64 pipe; the host lists
// only non-empty tiles.  Items with j = k copy the tile's own factor part.
template <typename T, bool PROJ>
__global__ void __launch_bounds__(128) k_blkdiag(const SlotDescT<T>* __restrict__ slots,
                                                 const BlkItem* __restrict__ items) {
  const BlkItem it = items[blockIdx.x];
  const SlotDescT<T> sd = slots[it.slot];
  const int j = it.j, a0 = 16 * it.rc, c0 = 16 * it.cc;
  const int nb = sd.nb, k = sd.k, i = sd.i;
  const int tid = threadIdx.x;
  const int C = PROJ ? sd.q : sd.bs;
  const int ldin = PROJ ? sd.r0 + sd.Ki : sd.ldx;          // P (project) or X (sample)
  const int ldout = PROJ ? sd.r0 + sd.Kk : sd.r0w + sd.Ki;  // Z (project) or W (sample)
  T* const outbase = PROJ ? sd.Z : sd.W;
  if (j == k) {  // leading block: the tile's own factor part
    const T* src = PROJ ? sd.P : sd.X0 + sd.x0off;
    const int lds = PROJ ? ldin : sd.ldx0;
    const int rows = PROJ ? sd.r0 : sd.r0w;  // rows past r0 (sample, padded layout) are zero
    for (int e = tid; e < 256; e += blockDim.x) {
      const int a = a0 + (e & 15), c = c0 + (e >> 4);
      if (a < rows && c < C) outbase[a + (size_t)c * ldout] = a < sd.r0 ? src[a + (size_t)c * lds] : T(0);
    }
    return;
  }
  const int rij = sd.rank[i * nb + j], rkj = sd.rank[k * nb + j];
  const int R = PROJ ? rkj : rij, K = PROJ ? rij : rkj;
  const T* Gij = sd.G + sd.goff[j] + (sd.voff[i * nb + j] - sd.voff[k * nb + j]);
  const int ldg = sd.gld[j];
  // sample: In = X_j (the r_kj rows of X at U_kj's offset); project: In = P_j (r_ij rows)
  const T* In = PROJ ? sd.P + sd.r0 + sd.uoff[i * nb + j] : sd.X + sd.uoff[k * nb + j];
  T* out = outbase + (PROJ ? sd.r0 + sd.uoff[k * nb + j] : sd.r0w + sd.uoff[i * nb + j]);
  __shared__ T As[16][17];  // op(G) chunk [row][kk]
  __shared__ T Bs[16][17];  // In chunk [kk][col]
  // Thread (row, column pair): warp w owns rows 4w .. 4w+3, so warps whose rows lie beyond R
  // skip the products, and the chunk loop stops at K: ranks are mostly well below 16, and
  // padded rows or depth would otherwise multiply the FP64 work.
  const int row = tid >> 3, cp = tid & 7;  // columns 2 cp, 2 cp + 1 of the tile
  const bool rows_live = a0 + 4 * (tid >> 5) < R;  // warp-uniform
  T acc0 = T(0), acc1 = T(0);
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int idx = tid + e * 128;
      int a, kk;
      if (PROJ) { kk = idx & 15; a = idx >> 4; }  // G_ij^T: consecutive threads walk a column of G
      else { a = idx & 15; kk = idx >> 4; }
      const int ga = a0 + a, gk = k0 + kk;
      As[a][kk] = (ga < R && gk < K) ? (PROJ ? Gij[gk + (size_t)ga * ldg] : Gij[ga + (size_t)gk * ldg]) : T(0);
      const int bk = idx & 15, bc = idx >> 4;
      Bs[bk][bc] = (k0 + bk < K && c0 + bc < C) ? In[(k0 + bk) + (size_t)(c0 + bc) * ldin] : T(0);
    }
    __syncthreads();
    if (rows_live) {
      const int kmax = min(16, K - k0);
      for (int kk = 0; kk < kmax; ++kk) {
        const T av = As[row][kk];
        acc0 = fma(av, Bs[kk][2 * cp], acc0);
        acc1 = fma(av, Bs[kk][2 * cp + 1], acc1);
      }
    }
    __syncthreads();
  }
  const int ga = a0 + row, gc = c0 + 2 * cp;
  if (ga < R) {
    if (gc < C) out[ga + (size_t)gc * ldout] = -acc0;
    if (gc + 1 < C) out[ga + (size_t)(gc + 1) * ldout] = -acc1;
  }
}

template <typename T>
void blkdiag_sample(tlr_ctx* ctx, const std::vector<BlkItem>& items, const SlotDescT<T>* slots_dev) {
  if (items.empty()) return;
  const BlkItem* it = static_cast<const BlkItem*>(upload(ctx, items.data(), items.size() * sizeof(BlkItem)));
  TLR_SITE_PRE(ctx);
  k_blkdiag<T, false><<<(unsigned)items.size(), 128, 0, ctx->stream>>>(slots_dev, it);
  TLR_LAUNCH_CHECK(ctx);
}
template <typename T>
void blkdiag_project(tlr_ctx* ctx, const std::vector<BlkItem>& items, const SlotDescT<T>* slots_dev) {
  if (items.empty()) return;
  const BlkItem* it = static_cast<const BlkItem*>(upload(ctx, items.data(), items.size() * sizeof(BlkItem)));
  TLR_SITE_PRE(ctx);
  k_blkdiag<T, true><<<(unsigned)items.size(), 128, 0, ctx->stream>>>(slots_dev, it);
  TLR_LAUNCH_CHECK(ctx);
}
template void blkdiag_sample<double>(tlr_ctx*, const std::vector<BlkItem>&, const SlotDescT<double>*);
template void blkdiag_sample<float>(tlr_ctx*, const std::vector<BlkItem>&, const SlotDescT<float>*);
template void blkdiag_project<double>(tlr_ctx*, const std::vector<BlkItem>&, const SlotDescT<double>*);
template void blkdiag_project<float>(tlr_ctx*, const std::vector<BlkItem>&, const SlotDescT<float>*);

// Batched Philox blocks: block g is Omega(seed_g, stream_g, k_g, t_g), b_g x bs, at out_g.
__global__ void k_omega_batched(const OmegaJob* __restrict__ jobs) {
  const OmegaJob J = jobs[blockIdx.y];
  const int n = J.b * J.bs;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; 2 * m < n; m += gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)m, J.t, J.k, J.stream};
    philox4x32_10(c, (uint32_t)J.seed, (uint32_t)(J.seed >> 32));
    const uint64_t a = ((uint64_t)c[1] << 32) | c[0];
    const uint64_t w = ((uint64_t)c[3] << 32) | c[2];
    const double u1 = ((double)(a >> 11) + 0.5) * 0x1p-53;
    const double u2 = (double)(w >> 11) * 0x1p-53 + 0x1p-54;
    const double rho = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    J.out[2 * m] = rho * cs;
    if (2 * m + 1 < n) J.out[2 * m + 1] = rho * sn;
  }
}
void omega_batched(tlr_ctx* ctx, std::vector<OmegaJob>& jobs) {
  if (jobs.empty()) return;
  int mx = 0;
  for (auto& j : jobs) mx = std::max(mx, j.b * j.bs);
  const OmegaJob* dj = static_cast<const OmegaJob*>(upload(ctx, jobs.data(), jobs.size() * sizeof(OmegaJob)));
  dim3 grid(std::min<unsigned>(cdiv((mx + 1) / 2, 256), 64u), (unsigned)jobs.size());
  TLR_SITE_PRE(ctx);
  k_omega_batched<<<grid, 256, 0, ctx->stream>>>(dj);
  TLR_LAUNCH_CHECK(ctx);
}

// Batched FP32 -> FP64 conversion.
__global__ void k_batched_to_double(const ConvBackJob* __restrict__ jobs) {
  const ConvBackJob J = jobs[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < J.n; e += (int64_t)gridDim.x * blockDim.x)
    J.dst[e] = (double)J.src[e];
}
void batched_to_double(tlr_ctx* ctx, std::vector<ConvBackJob>& jobs) {
  std::vector<ConvBackJob> nz;
  int64_t mx = 0;
  for (auto& j : jobs)
    if (j.n > 0) { nz.push_back(j); mx = std::max(mx, j.n); }
  for (size_t o = 0; o < nz.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, nz.size() - o);
    const ConvBackJob* dj = static_cast<const ConvBackJob*>(upload(ctx, nz.data() + o, cnt * sizeof(ConvBackJob)));
    dim3 grid(std::min<unsigned>(cdiv(mx, 256), 64u), (unsigned)cnt);
    TLR_SITE_PRE(ctx);
    k_batched_to_double<<<grid, 256, 0, ctx->stream>>>(dj);
    TLR_LAUNCH_CHECK(ctx);
  }
}

// Batched row scaling Y = diag(d)^{+-1} X (LDL^T: D_j V_kj, and V = D^{-1} L^{-1} B).
__global__ void k_batched_scale_rows(const ScaleJob* __restrict__ jobs) {
  const ScaleJob J = jobs[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)J.m * J.n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % J.m), c = (int)(e / J.m);
    const double s = J.inv ? 1.0 / J.d[r] : J.d[r];
    J.Y[r + (size_t)c * J.ldy] = J.X[r + (size_t)c * J.ldx] * s;
  }
}
void batched_scale_rows(tlr_ctx* ctx, std::vector<ScaleJob>& jobs) {
  std::vector<ScaleJob> nz;
  int64_t mx = 0;
  for (auto& j : jobs)
    if ((int64_t)j.m * j.n > 0) { nz.push_back(j); mx = std::max(mx, (int64_t)j.m * j.n); }
  for (size_t o = 0; o < nz.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, nz.size() - o);
    const ScaleJob* dj = static_cast<const ScaleJob*>(upload(ctx, nz.data() + o, cnt * sizeof(ScaleJob)));
    dim3 grid(std::min<unsigned>(cdiv(mx, 256), 128u), (unsigned)cnt);
    TLR_SITE_PRE(ctx);
    k_batched_scale_rows<<<grid, 256, 0, ctx->stream>>>(dj);
    TLR_LAUNCH_CHECK(ctx);
  }
}

// Batched diagonal shift A_ii += s.
__global__ void k_batched_add_diag(const DiagJob* __restrict__ jobs) {
  const DiagJob J = jobs[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.n; i += gridDim.x * blockDim.x)
    J.A[i + (size_t)i * J.lda] += J.s;
}
void batched_add_diag(tlr_ctx* ctx, std::vector<DiagJob>& jobs) {
  if (jobs.empty()) return;
  int mx = 0;
  for (auto& j : jobs) mx = std::max(mx, j.n);
  for (size_t o = 0; o < jobs.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, jobs.size() - o);
    const DiagJob* dj = static_cast<const DiagJob*>(upload(ctx, jobs.data() + o, cnt * sizeof(DiagJob)));
    dim3 grid(std::min<unsigned>(cdiv(mx, 256), 16u), (unsigned)cnt);
    TLR_SITE_PRE(ctx);
    k_batched_add_diag<<<grid, 256, 0, ctx->stream>>>(dj);
    TLR_LAUNCH_CHECK(ctx);
  }
}

// ------------------------------------------------------------------ FP64 peak probe
__global__ void k_dfma_loop(double* out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

double fp64_peak(tlr_ctx* ctx) {
  const int blocks = ctx->sm_count * 4, threads = 256, iters = 4096;
  double* d = static_cast<double*>(dalloc(ctx, sizeof(double) * blocks * threads));
  cudaEvent_t e0, e1;
  TLR_CUDA(cudaEventCreate(&e0));
  TLR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    TLR_CUDA(cudaEventRecord(e0, ctx->stream));
    TLR_SITE_PRE(ctx);
    k_dfma_loop<<<blocks, threads, 0, ctx->stream>>>(d, iters, 0.9999, 1e-3);
    TLR_LAUNCH_CHECK(ctx);
    TLR_CUDA(cudaEventRecord(e1, ctx->stream));
    TLR_CUDA(cudaEventSynchronize(e1));
    float ms;
    TLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(ctx, d);
  return 2.0 * 8 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
}

// ------------------------------------------------------------------ batched copies (updateTiles)
__global__ void k_batched_copy(const CopyJob* __restrict__ jobs, int njobs) {
  const CopyJob J = jobs[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < J.n; e += (int64_t)gridDim.x * blockDim.x)
    J.dst[e] = J.src[e];
}
void batched_copy(tlr_ctx* ctx, std::vector<CopyJob>& jobs) {
  std::vector<CopyJob> nz;
  int64_t mx = 0;
  for (auto& j : jobs)
    if (j.n > 0) { nz.push_back(j); mx = std::max(mx, j.n); }
  for (size_t o = 0; o < nz.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, nz.size() - o);
    const CopyJob* dj = static_cast<const CopyJob*>(upload(ctx, nz.data() + o, cnt * sizeof(CopyJob)));
    dim3 grid(std::min<unsigned>(cdiv(mx, 256), 64u), (unsigned)cnt);
    TLR_SITE_PRE(ctx);
    k_batched_copy<<<grid, 256, 0, ctx->stream>>>(dj, cnt);
    TLR_LAUNCH_CHECK(ctx);
  }
}

__global__ void k_scale_cols(int m, int n, const double* __restrict__ dv, const double* X, int ldx,
                             double* Y, int ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    Y[r + (size_t)c * ldy] = X[r + (size_t)c * ldx] * dv[c];
  }
}
void scale_cols(tlr_ctx* ctx, int m, int n, const double* dvec, const double* X, int ldx, double* Y,
                int ldy) {
  if ((int64_t)m * n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_scale_cols<<<std::min<unsigned>(cdiv((int64_t)m * n, 256), 4096u), 256, 0, ctx->stream>>>(m, n, dvec, X,
                                                                                             ldx, Y, ldy);
  TLR_LAUNCH_CHECK(ctx);
}

// Zero the strict upper triangle (and set a unit diagonal if `unit`).
__global__ void k_tril_mask(int n, double* A, int lda, int unit) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    if (r < c) A[r + (size_t)c * lda] = 0.0;
    else if (r == c && unit) A[r + (size_t)c * lda] = 1.0;
  }
}
void tril_mask(tlr_ctx* ctx, int n, double* A, int lda, int unit) {
  if (n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_tril_mask<<<std::min<unsigned>(cdiv((int64_t)n * n, 256), 4096u), 256, 0, ctx->stream>>>(n, A, lda, unit);
  TLR_LAUNCH_CHECK(ctx);
}

__global__ void k_set_diag(int n, double* A, int lda, const double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + (size_t)i * lda] = d[i];
}
void set_diag(tlr_ctx* ctx, int n, double* A, int lda, const double* d) {
  if (n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_set_diag<<<cdiv(n, 256), 256, 0, ctx->stream>>>(n, A, lda, d);
  TLR_LAUNCH_CHECK(ctx);
}

// Y += alpha X (m x n).
__global__ void k_axpy_matrix(int m, int n, double alpha, const double* __restrict__ X, int ldx, double* Y, int ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    Y[r + (size_t)c * ldy] += alpha * X[r + (size_t)c * ldx];
  }
}
void axpy_matrix(tlr_ctx* ctx, int m, int n, double alpha, const double* X, int ldx, double* Y, int ldy) {
  if ((int64_t)m * n <= 0) return;
  TLR_SITE_PRE(ctx);
  k_axpy_matrix<<<std::min<unsigned>(cdiv((int64_t)m * n, 256), 4096u), 256, 0, ctx->stream>>>(m, n, alpha, X, ldx,
                                                                                              Y, ldy);
  TLR_LAUNCH_CHECK(ctx);
}

// Batched FP64 -> FP32 conversion of contiguous ranges (FP32 operands of the sampling chains).
__global__ void k_batched_to_float(const ConvJob* __restrict__ jobs) {
  const ConvJob J = jobs[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < J.n; e += (int64_t)gridDim.x * blockDim.x)
    J.dst[e] = (float)J.src[e];
}
void batched_to_float(tlr_ctx* ctx, std::vector<ConvJob>& jobs) {
  std::vector<ConvJob> nz;
  int64_t mx = 0;
  for (auto& j : jobs)
    if (j.n > 0) { nz.push_back(j); mx = std::max(mx, j.n); }
  for (size_t o = 0; o < nz.size(); o += 65535) {
    const int cnt = (int)std::min<size_t>(65535, nz.size() - o);
    const ConvJob* dj = static_cast<const ConvJob*>(upload(ctx, nz.data() + o, cnt * sizeof(ConvJob)));
    dim3 grid(std::min<unsigned>(cdiv(mx, 256), 64u), (unsigned)cnt);
    TLR_SITE_PRE(ctx);
    k_batched_to_float<<<grid, 256, 0, ctx->stream>>>(dj);
    TLR_LAUNCH_CHECK(ctx);
  }
}

// Squared 2-norms of the columns of a column-major rows x ncols matrix (one warp per column).
__global__ void k_col_sqnorms(const double* __restrict__ X, int rows, int64_t ncols, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (c >= ncols) return;
  const double* x = X + (size_t)c * rows;
  double s = 0.0;
  for (int r = lane; r < rows; r += 32) s = fma(x[r], x[r], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}
void col_sqnorms(tlr_ctx* ctx, const double* X, int rows, int64_t ncols, double* out) {
  if (ncols <= 0) return;
  TLR_SITE_PRE(ctx);
  k_col_sqnorms<<<cdiv(ncols, 8), 256, 0, ctx->stream>>>(X, rows, ncols, out);
  TLR_LAUNCH_CHECK(ctx);
}

}  // namespace tlr
