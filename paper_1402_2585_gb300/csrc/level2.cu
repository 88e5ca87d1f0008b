// Blocked second coarsening of the little Dirac operator (three-level HDCG).
//
// The little Dirac operator A is itself a nearest-neighbour operator on the
// coarse lattice (an 81-point stencil, Sec. 5.1), so the construction of
// Sec. 2 applies to it once more:
//  * Nvec2 coarse vectors phi2_k are cut into 4D blocks of the coarse lattice
//    and the block pieces are orthonormalised (two rounds of Cholesky QR with
//    FP64 Gram matrices);
//  * R2 c = <phi2^b, c>, P2 = R2^dag;
//  * A2 = P2^dag A P2, contracted directly from the blocks of A in FP64: A
//    reaches one coarse site, so A2 couples a level-2 block only to blocks at
//    most one hop away and is again an 81-point stencil (canonical layout,
//    the aliasing rule of hdcg.h for level-2 extents 1 and 2);
//  * the level-1 solve (the coarse-grid correction Q = P A^-1 R of the fine
//    A-DEF2) is A-DEF2 on A with Q2 = P2 A2^-1 R2 -- Fig. pcg_general and
//    Table algos one level down -- with M = 1 as the smoother:
//      x0 = Q2 b, y = M1 r = r + Q2 (r - A r), flexible (Polak-Ribiere) beta;
//  * A2^-1 is a dense matrix: the level-2 operator is small (Vc2 * Nvec2
//    unknowns, 12,288 for 32^3 x 64 with 4^4 then 2^4 blocks and Nvec 40 then
//    24), so its inverse is formed once by blocked Gauss-Jordan elimination
//    (Jacobi-scaled; pivot blocks inverted in FP64) and applied as one
//    matrix product per level-1 iteration, the analogue of the paper's dense
//    prediagonalised coarsest level (Sec. 5.2).
// Vectors of the level-1 solve are FP32 [e][r] (e = a * Nvec + j, right-hand
// side fastest), as in the other multi-right-hand-side coarse solvers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "coarse.cuh"

namespace hdcg {

__global__ void k_cholinv(const double2* G, double2* T, int n, size_t Vc, int* fail);  // coarse.cu

namespace {

constexpr int L2_MAXV = 64;   // largest Nvec2 (and Nvec of the level-1 operator)

unsigned nblocks(size_t n) { return (unsigned)((n + 255) / 256); }

void smem_limit(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) HDCG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// offset along one dimension of extent L between block coordinates (difference
// d), in the canonical storage: -1/0/+1 for L >= 3, 0/+1 for L = 2 (-1 is +1),
// 0 for L = 1; -2 for blocks more than one hop apart
__host__ __device__ inline int canon_delta(int d, int L) {
  d = ((d % L) + L) % L;
  if (L == 1) return 0;
  if (L == 2) return d;
  if (d == 0) return 0;
  if (d == 1) return 1;
  if (d == L - 1) return -1;
  return -2;
}

// offsets stored along an extent L (hdcg.h)
bool kept(int d, int L) { return L >= 3 ? true : (L == 2 ? d >= 0 : d == 0); }

// ---------------------------------------------------------------------------
// block orthonormalisation of the level-2 vectors
// ---------------------------------------------------------------------------

// G[b][j][k] = sum over the coarse sites a of block b and m < n1 of
// conj(phi_j[a][m]) phi_k[a][m], FP64 products; one CTA per block
__global__ void __launch_bounds__(256) k_l2_gram(const float2* __restrict__ phi, size_t ne, int nv, int n1,
                                                 const int* __restrict__ sites, int spb, double2* G) {
  extern __shared__ float2 sv[];   // [nv][n1]: all vectors at one coarse site
  const int b = blockIdx.x;
  const int npair = nv * nv;
  double gr[16], gi[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) gr[q] = gi[q] = 0.0;
  for (int i = 0; i < spb; ++i) {
    const size_t a = (size_t)sites[(size_t)b * spb + i];
    __syncthreads();
    for (int q = threadIdx.x; q < nv * n1; q += blockDim.x) {
      const int k = q / n1, m = q % n1;
      sv[q] = phi[(size_t)k * ne + a * n1 + m];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p = threadIdx.x + q * blockDim.x;
      if (p < npair) {
        const int j = p / nv, k = p % nv;
        double sr = 0, si = 0;
        for (int m = 0; m < n1; ++m) {
          const float2 x = sv[j * n1 + m], y = sv[k * n1 + m];
          sr += (double)x.x * y.x + (double)x.y * y.y;
          si += (double)x.x * y.y - (double)x.y * y.x;
        }
        gr[q] += sr;
        gi[q] += si;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p = threadIdx.x + q * blockDim.x;
    if (p < npair) G[(size_t)b * npair + p] = make_double2(gr[q], gi[q]);
  }
}

// phi_k[e] <- sum_{j <= k} phi_j[e] T[b(e)][j][k] (T upper triangular), one thread per unknown e
__global__ void k_l2_transform(float2* phi, size_t ne, int nv, int n1, const int* __restrict__ blk,
                               const double2* __restrict__ T) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double2* t = T + (size_t)blk[e / n1] * nv * nv;
  double2 v[L2_MAXV];
  for (int j = 0; j < nv; ++j) {
    const float2 f = phi[(size_t)j * ne + e];
    v[j] = make_double2(f.x, f.y);
  }
  for (int k = 0; k < nv; ++k) {
    double sr = 0, si = 0;
    for (int j = 0; j <= k; ++j) {
      const double2 q = t[j * nv + k];
      sr += v[j].x * q.x - v[j].y * q.y;
      si += v[j].x * q.y + v[j].y * q.x;
    }
    phi[(size_t)k * ne + e] = make_float2((float)sr, (float)si);
  }
}

// ---------------------------------------------------------------------------
// R2, P2 (several right-hand sides, coarse vectors [e][r], level-2 vectors [i][r])
// ---------------------------------------------------------------------------

// c2[b][k][r] = sum_{a in b, m} conj(phi_k[a][m]) (x - xs)[a n1 + m][r]; xs may be null.
// One CTA per level-2 block; up to 4 outputs (k, r) per thread (nv * R <= 1024).
__global__ void __launch_bounds__(256) k_l2_restrict(const float2* __restrict__ phi, size_t ne, int nv, int n1,
                                                     const int* __restrict__ sites, int spb,
                                                     const float2* __restrict__ x, const float2* __restrict__ xs,
                                                     int R, float2* c2, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ float2 sm[];
  float2* xv = sm;             // [n1][R]
  float2* pv = sm + n1 * R;    // [nv][n1]
  const int b = blockIdx.x;
  const int nout = nv * R;
  float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = 0; i < spb; ++i) {
    const size_t a = (size_t)sites[(size_t)b * spb + i];
    __syncthreads();
    for (int q = threadIdx.x; q < n1 * R; q += blockDim.x) {
      float2 v = x[a * n1 * R + q];
      if (xs) {
        const float2 s = xs[a * n1 * R + q];
        v.x -= s.x;
        v.y -= s.y;
      }
      xv[q] = v;
    }
    for (int q = threadIdx.x; q < nv * n1; q += blockDim.x) {
      const int k = q / n1, m = q % n1;
      pv[q] = phi[(size_t)k * ne + a * n1 + m];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = threadIdx.x + u * blockDim.x;
      if (o < nout) {
        const int k = o / R, r = o % R;
        for (int m = 0; m < n1; ++m) {
          const float2 p = pv[k * n1 + m], v = xv[m * R + r];
          ar[u] += p.x * v.x + p.y * v.y;
          ai[u] += p.x * v.y - p.y * v.x;
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int o = threadIdx.x + u * blockDim.x;
    if (o < nout) c2[(size_t)b * nout + o] = make_float2(ar[u], ai[u]);
  }
}

// y[e][r] = (add ? add[e][r] : 0) + sum_k phi_k[e] c2[b(e)][k][r]; with want_dot the
// per-right-hand-side Re<dv, y> is reduced (dv = r in the level-1 solver: (r, y))
__global__ void __launch_bounds__(256) k_l2_prolong(const float2* __restrict__ phi, size_t ne, int nv, int n1,
                                                    const int* __restrict__ blk, const float2* __restrict__ c2,
                                                    int R, const float2* __restrict__ add, float2* y,
                                                    const int* skip, Reduction red, int want_dot,
                                                    const float2* __restrict__ dv) {
  if (skip && *skip) return;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float ar[RMAX], ai[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) ar[q] = ai[q] = 0.f;
  double v[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) v[q] = 0.0;
  if (e < ne) {
    const float2* cb = c2 + (size_t)blk[e / n1] * nv * R;
    for (int k = 0; k < nv; ++k) {
      const float2 p = phi[(size_t)k * ne + e];
#pragma unroll
      for (int q = 0; q < RMAX; ++q)
        if (q < R) {
          const float2 cv = cb[k * R + q];
          ar[q] += p.x * cv.x - p.y * cv.y;
          ai[q] += p.x * cv.y + p.y * cv.x;
        }
    }
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        float2 o = make_float2(ar[q], ai[q]);
        if (add) {
          const float2 s = add[e * R + q];
          o.x += s.x;
          o.y += s.y;
        }
        if (want_dot) {
          const float2 s = dv[e * R + q];
          v[q] = (double)s.x * o.x + (double)s.y * o.y;
        }
        y[e * R + q] = o;
      }
  }
  if (want_dot) grid_reduce<RMAX>(v, red, R);
}

// u[i][r] = sum_j M[i][j] t[j][r]: dense level-2 inverse, one warp per row
template <typename MT>
__global__ void __launch_bounds__(256) k_dense_apply(const MT* __restrict__ M, size_t N,
                                                     const float2* __restrict__ t, int R, float2* u,
                                                     const int* skip) {
  if (skip && *skip) return;
  using RT = decltype(MT{}.x);
  const size_t row = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  RT ar[RMAX], ai[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) ar[q] = ai[q] = 0;
  const MT* m = M + row * N;
  for (size_t j = lane; j < N; j += 32) {
    const MT a = m[j];
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const float2 tv = t[j * R + q];
        ar[q] += a.x * (RT)tv.x - a.y * (RT)tv.y;
        ai[q] += a.x * (RT)tv.y + a.y * (RT)tv.x;
      }
  }
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    if (q >= R) break;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[q] += __shfl_xor_sync(FULL_MASK, ar[q], o);
      ai[q] += __shfl_xor_sync(FULL_MASK, ai[q], o);
    }
    if (lane == 0) u[row * R + q] = make_float2((float)ar[q], (float)ai[q]);
  }
}

// ---------------------------------------------------------------------------
// A2 = P2^dag A P2 (FP64), one CTA per coarse site a:
//   A2[b(a)][l2][J][K] += sum_l sum_{m,n} conj(phi_J[a][m]) A[a][l][m][n] phi_K[a'][n],
// a' = a + delta_l, l2 the canonical level-2 offset from b(a) to b(a').  A is in
// the internal layout (block (a, l) stored transposed: element (m, n) at [n][m]).
// ---------------------------------------------------------------------------
template <typename AT>
__device__ __forceinline__ double2 ld_entry(const AT* p);
template <> __device__ __forceinline__ double2 ld_entry<double2>(const double2* p) { return *p; }
template <> __device__ __forceinline__ double2 ld_entry<float2>(const float2* p) {
  const float2 v = *p;
  return make_double2(v.x, v.y);
}

template <typename AT>
__global__ void __launch_bounds__(256) k_l2_galerkin(const AT* __restrict__ A, const int* __restrict__ cnbr, int n1,
                                                     const unsigned* __restrict__ keep_mask,
                                                     const float2* __restrict__ phi, size_t ne, int nv,
                                                     const int* __restrict__ blk, const int* __restrict__ coords2,
                                                     int4 L2, double2* A2, int* err) {
  extern __shared__ double2 dsm[];
  double2* Ab = dsm;                          // [n1][n1]  (m, n)
  double2* T1 = Ab + n1 * n1;                 // [n1][nv]  sum_n A[m][n] phi_K[a'][n]
  float2* pa = reinterpret_cast<float2*>(T1 + n1 * nv);   // [nv][n1] phi at a
  float2* pb = pa + nv * n1;                  // [nv][n1] phi at a'
  const size_t a = blockIdx.x;
  const int b = blk[a];
  for (int q = threadIdx.x; q < nv * n1; q += blockDim.x) {
    const int k = q / n1, m = q % n1;
    pa[q] = phi[(size_t)k * ne + a * n1 + m];
  }
  for (int l = 0; l < 81; ++l) {
    if (!((keep_mask[l >> 5] >> (l & 31)) & 1u)) continue;
    const size_t a2 = (size_t)cnbr[a * 81 + l];
    const int bb = blk[a2];
    int l2 = 0, mul = 1;
    bool ok = true;
    const int Ls2[4] = {L2.x, L2.y, L2.z, L2.w};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int d = canon_delta(coords2[bb * 4 + mu] - coords2[b * 4 + mu], Ls2[mu]);
      if (d < -1) ok = false;
      l2 += (d + 1) * mul;
      mul *= 3;
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      continue;
    }
    __syncthreads();
    const AT* blkA = A + ((size_t)a * 81 + l) * n1 * n1;
    for (int q = threadIdx.x; q < n1 * n1; q += blockDim.x) {
      const int n = q / n1, m = q % n1;   // stored [n][m]
      Ab[m * n1 + n] = ld_entry<AT>(blkA + q);
    }
    for (int q = threadIdx.x; q < nv * n1; q += blockDim.x) {
      const int k = q / n1, m = q % n1;
      pb[q] = phi[(size_t)k * ne + a2 * n1 + m];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n1 * nv; q += blockDim.x) {
      const int m = q / nv, K = q % nv;
      double sr = 0, si = 0;
      for (int n = 0; n < n1; ++n) {
        const double2 x = Ab[m * n1 + n];
        const float2 y = pb[K * n1 + n];
        sr += x.x * y.x - x.y * y.y;
        si += x.x * y.y + x.y * y.x;
      }
      T1[q] = make_double2(sr, si);
    }
    __syncthreads();
    double2* out = A2 + ((size_t)b * 81 + l2) * nv * nv;
    for (int q = threadIdx.x; q < nv * nv; q += blockDim.x) {
      const int J = q / nv, K = q % nv;
      double sr = 0, si = 0;
      for (int m = 0; m < n1; ++m) {
        const float2 x = pa[J * n1 + m];   // conj(x) * T1
        const double2 y = T1[m * nv + K];
        sr += x.x * y.x + x.y * y.y;
        si += x.x * y.y - x.y * y.x;
      }
      atomicAdd(&out[q].x, sr);
      atomicAdd(&out[q].y, si);
    }
  }
}

// ---------------------------------------------------------------------------
// dense inverse by blocked Gauss-Jordan elimination (in place, no pivoting: the
// Jacobi-scaled A2 is Hermitian positive definite).  Step k, pivot block K of
// GJB rows/columns:  P = M[K][K]^-1;  M[i][K] <- M[i][K] P;
// M[i][j] <- M[i][j] - M[i][K] M[K][j] (old row K);  M[K][j] <- -P M[K][j];
// M[K][K] <- P  (i, j outside K).  After the last step M holds the inverse.
// ---------------------------------------------------------------------------
constexpr int GJB = 32;

// D = the scaled dense level-2 matrix: M[i][j] = A2_ij s_i s_j, s_i = 1/sqrt(Re A2_ii)
template <typename MT>
__global__ void k_l2_dense(const double2* __restrict__ A2, const int* __restrict__ cnbr2,
                           const unsigned* __restrict__ keep_mask, int nv, size_t Vc2, const double* __restrict__ s,
                           MT* M) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)81 * nv * nv;
  if (t >= Vc2 * per) return;
  const size_t b = t / per;
  const int rem = (int)(t % per);
  const int l = rem / (nv * nv), J = (rem / nv) % nv, K = rem % nv;
  if (!((keep_mask[l >> 5] >> (l & 31)) & 1u)) return;
  const size_t N = Vc2 * nv;
  const size_t row = b * nv + J, col = (size_t)cnbr2[b * 81 + l] * nv + K;
  const double2 v = A2[t];
  const double f = s[row] * s[col];
  M[row * N + col] = {(decltype(MT{}.x))(v.x * f), (decltype(MT{}.x))(v.y * f)};
}

__global__ void k_l2_scale(const double2* __restrict__ A2, int nv, size_t Vc2, double* s, int* err) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Vc2 * nv) return;
  const size_t b = t / nv;
  const int J = (int)(t % nv);
  const double d = A2[((b * 81 + 40) * nv + J) * nv + J].x;   // l = 40: offset 0
  if (!(d > 0.0)) atomicExch(err, 1);
  s[t] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
}

// Minv[i][j] <- Minv[i][j] s_i s_j
template <typename MT>
__global__ void k_l2_unscale(MT* M, size_t N, const double* __restrict__ s) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * N) return;
  const double f = s[t / N] * s[t % N];
  MT v = M[t];
  v.x = (decltype(v.x))(v.x * f);
  v.y = (decltype(v.y))(v.y * f);
  M[t] = v;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// pivot block: P = M[K][K]^-1 by unblocked Gauss-Jordan in FP64 (one CTA); P is
// written to Pbuf (FP64) and to M[K][K]
template <typename MT>
__global__ void __launch_bounds__(256) k_gj_pivot(MT* M, size_t N, size_t k0, int nb, double2* Pbuf, int* err) {
  __shared__ double2 D[GJB][GJB + 1];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int i = q / nb, j = q % nb;
    const MT v = M[(k0 + i) * N + k0 + j];
    D[i][j] = make_double2(v.x, v.y);
  }
  __syncthreads();
  for (int p = 0; p < nb; ++p) {
    const double2 dp = D[p][p];
    const double den = dp.x * dp.x + dp.y * dp.y;
    if (!(den > 0.0) || !(den < 1e300)) {
      if (threadIdx.x == 0) atomicExch(err, 2);
    }
    const double2 piv = den > 0.0 ? make_double2(dp.x / den, -dp.y / den) : make_double2(0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      if (i != p) D[i][p] = cmul(D[i][p], piv);
    __syncthreads();
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
      const int i = q / nb, j = q % nb;
      if (i != p && j != p) {
        const double2 u = cmul(D[i][p], D[p][j]);
        D[i][j].x -= u.x;
        D[i][j].y -= u.y;
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      if (j != p) {
        const double2 u = cmul(piv, D[p][j]);
        D[p][j] = make_double2(-u.x, -u.y);
      } else {
        D[p][p] = piv;
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int i = q / nb, j = q % nb;
    Pbuf[q] = D[i][j];
    M[(k0 + i) * N + k0 + j] = {(decltype(MT{}.x))D[i][j].x, (decltype(MT{}.x))D[i][j].y};
  }
}

// column panel: M[i][K] <- M[i][K] P for rows i outside K; one warp per row
template <typename MT>
__global__ void __launch_bounds__(256) k_gj_col(MT* M, size_t N, size_t k0, int nb, const double2* __restrict__ Pbuf) {
  __shared__ double2 P[GJB][GJB + 1];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) P[q / nb][q % nb] = Pbuf[q];
  __syncthreads();
  const size_t i = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= N || (i >= k0 && i < k0 + nb)) return;
  double2 v = make_double2(0, 0);
  if (lane < nb) {
    const MT m = M[i * N + k0 + lane];
    v = make_double2(m.x, m.y);
  }
  double2 o = make_double2(0, 0);
  for (int q = 0; q < nb; ++q) {
    const double2 mq = make_double2(__shfl_sync(FULL_MASK, v.x, q), __shfl_sync(FULL_MASK, v.y, q));
    if (lane < nb) {
      const double2 u = cmul(mq, P[q][lane]);
      o.x += u.x;
      o.y += u.y;
    }
  }
  if (lane < nb) M[i * N + k0 + lane] = {(decltype(MT{}.x))o.x, (decltype(MT{}.x))o.y};
}

// trailing update: M[i][j] -= sum_q M[i][k0 + q] M[k0 + q][j] for i, j outside K;
// 64 x 64 tiles, 4 x 4 outputs per thread
template <typename MT>
__global__ void __launch_bounds__(256) k_gj_update(MT* M, size_t N, size_t k0, int nb) {
  using RT = decltype(MT{}.x);
  extern __shared__ unsigned char gsm[];
  MT* Lt = reinterpret_cast<MT*>(gsm);            // [64][GJB + 1]
  MT* Ut = Lt + 64 * (GJB + 1);                   // [GJB][64 + 1]
  const size_t i0 = (size_t)blockIdx.y * 64, j0 = (size_t)blockIdx.x * 64;
  for (int q = threadIdx.x; q < 64 * GJB; q += blockDim.x) {
    const int r = q / GJB, c = q % GJB;
    const size_t i = i0 + r;
    Lt[r * (GJB + 1) + c] = (i < N && c < nb) ? M[i * N + k0 + c] : MT{0, 0};
  }
  for (int q = threadIdx.x; q < GJB * 64; q += blockDim.x) {
    const int r = q / 64, c = q % 64;
    const size_t j = j0 + c;
    Ut[r * 65 + c] = (j < N && r < nb) ? M[(k0 + r) * N + j] : MT{0, 0};
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  RT cr[4][4], ci[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) cr[u][w] = ci[u][w] = 0;
  for (int q = 0; q < nb; ++q) {
    MT lv[4], uv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) lv[u] = Lt[(ty * 4 + u) * (GJB + 1) + q];
#pragma unroll
    for (int w = 0; w < 4; ++w) uv[w] = Ut[q * 65 + tx + 16 * w];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        cr[u][w] += lv[u].x * uv[w].x - lv[u].y * uv[w].y;
        ci[u][w] += lv[u].x * uv[w].y + lv[u].y * uv[w].x;
      }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const size_t i = i0 + ty * 4 + u;
    if (i >= N || (i >= k0 && i < k0 + nb)) continue;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const size_t j = j0 + tx + 16 * w;
      if (j >= N || (j >= k0 && j < k0 + nb)) continue;
      MT v = M[i * N + j];
      v.x -= cr[u][w];
      v.y -= ci[u][w];
      M[i * N + j] = v;
    }
  }
}

// row panel: M[K][j] <- -P M[K][j] for columns j outside K; 32 columns per CTA
template <typename MT>
__global__ void __launch_bounds__(256) k_gj_row(MT* M, size_t N, size_t k0, int nb, const double2* __restrict__ Pbuf) {
  __shared__ double2 P[GJB][GJB + 1];
  __shared__ double2 T[GJB][33];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) P[q / nb][q % nb] = Pbuf[q];
  const size_t j0 = (size_t)blockIdx.x * 32;
  for (int q = threadIdx.x; q < GJB * 32; q += blockDim.x) {
    const int r = q / 32, c = q % 32;
    const size_t j = j0 + c;
    if (r < nb && j < N) {
      const MT v = M[(k0 + r) * N + j];
      T[r][c] = make_double2(v.x, v.y);
    } else {
      T[r][c] = make_double2(0, 0);
    }
  }
  __syncthreads();
  const int c = threadIdx.x % 32, r0 = threadIdx.x / 32;
  const size_t j = j0 + c;
  if (j >= N || (j >= k0 && j < k0 + nb)) return;
  for (int r = r0; r < nb; r += 8) {
    double sr = 0, si = 0;
    for (int p = 0; p < nb; ++p) {
      const double2 u = cmul(P[r][p], T[p][c]);
      sr += u.x;
      si += u.y;
    }
    M[(k0 + r) * N + j] = {(decltype(MT{}.x))(-sr), (decltype(MT{}.x))(-si)};
  }
}

template <typename MT>
void gj_inverse(Ctx& c, MT* M, size_t N, double2* Pbuf, int* err) {
  const size_t smem = (size_t)(64 * (GJB + 1) + GJB * 65) * sizeof(MT);
  smem_limit((const void*)k_gj_update<MT>, smem);
  const dim3 gu((unsigned)((N + 63) / 64), (unsigned)((N + 63) / 64));
  for (size_t k0 = 0; k0 < N; k0 += GJB) {
    const int nb = (int)std::min<size_t>(GJB, N - k0);
    k_gj_pivot<MT><<<1, 256, 0, c.stream>>>(M, N, k0, nb, Pbuf, err);
    k_gj_col<MT><<<(unsigned)((N + 7) / 8), 256, 0, c.stream>>>(M, N, k0, nb, Pbuf);
    k_gj_update<MT><<<gu, 256, smem, c.stream>>>(M, N, k0, nb);
    k_gj_row<MT><<<(unsigned)((N + 31) / 32), 256, 0, c.stream>>>(M, N, k0, nb, Pbuf);
    HDCG_CUDA(cudaGetLastError());
    c.launches += 4;
  }
}

// ---------------------------------------------------------------------------
// the level-1 A-DEF2 iteration
// ---------------------------------------------------------------------------
struct CtlL2 {
  double bb[RMAX];
  double rr[RMAX];          // |r|^2 ...
  double ryo[RMAX];         // ... and (r_new, y_old): one reduction of 2 RMAX values
  double pAp[RMAX];
  double ry[2][RMAX];       // (r, y) by parity
  double stop[RMAX];
  int done[RMAX];
  unsigned xm[3][RMAX];     // max |Re|, |Im| of p (0), r (1) and M r (2): tensor-core operand scales
  int iter;
  int all_done;
  int broke;                // a right-hand side stopped on (p, A p) <= 0 or a NaN above its tolerance
};

// |b|^2 per right-hand side; x = 0 elsewhere is set by the prolongation of Q2 b
__global__ void k_l1_norm(const float2* __restrict__ v, size_t ne, int R, Reduction red) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) s[q] = 0.0;
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const float2 a = v[t * R + q];
        s[q] = (double)a.x * a.x + (double)a.y * a.y;
      }
  grid_reduce<RMAX>(s, red, R);
}

__device__ __forceinline__ void warp_max_to(float m, unsigned* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(dst, __float_as_uint(m));
}

// v = a - b (per element), |v|^2 per rhs, max|v| into xm (cleared beforehand)
__global__ void k_l1_residual(const float2* __restrict__ a, const float2* __restrict__ b, float2* v, size_t ne, int R,
                              unsigned* xm, Reduction red) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[RMAX];
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    s[q] = 0.0;
    m[q] = 0.f;
  }
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const float2 x = a[t * R + q], y = b[t * R + q];
        const float2 d = make_float2(x.x - y.x, x.y - y.y);
        v[t * R + q] = d;
        s[q] = (double)d.x * d.x + (double)d.y * d.y;
        m[q] = fmaxf(fabsf(d.x), fabsf(d.y));
      }
#pragma unroll
  for (int q = 0; q < RMAX; ++q)
    if (q < R) warp_max_to(m[q], xm + q);
  grid_reduce<RMAX>(s, red, R);
}

__global__ void k_l1_start(CtlL2* ctl, int R, double tol, int maxiter) {
  int all = 1;
  for (int q = 0; q < RMAX; ++q) {
    ctl->stop[q] = q < R ? tol * tol * ctl->bb[q] : 0.0;
    ctl->done[q] = q < R ? ((ctl->bb[q] == 0.0 || ctl->rr[q] <= ctl->stop[q] || maxiter <= 0) ? 1 : 0) : 1;
    all &= ctl->done[q];
    ctl->xm[0][q] = 0u;
  }
  ctl->iter = 0;
  ctl->all_done = all;
}

// p = y (first) or y + beta p (flexible beta); max|p| into xm[0]; clears xm[1]
__global__ void k_l1_p(float2* p, const float2* __restrict__ y, size_t ne, int R, CtlL2* ctl, int par, int first) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < RMAX) ctl->xm[1][t] = 0u;
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) m[q] = 0.f;
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const size_t o = t * R + q;
        float2 pv = p[o];
        if (!ctl->done[q]) {
          float beta = 0.f;
          if (!first) {
            const double ro = ctl->ry[par][q];
            beta = (float)(ro != 0.0 ? (ctl->ry[par ^ 1][q] - ctl->ryo[q]) / ro : 0.0);
          }
          const float2 yv = y[o];
          pv.x = yv.x + beta * pv.x;
          pv.y = yv.y + beta * pv.y;
          p[o] = pv;
        }
        m[q] = fmaxf(fabsf(pv.x), fabsf(pv.y));
      }
#pragma unroll
  for (int q = 0; q < RMAX; ++q)
    if (q < R) warp_max_to(m[q], ctl->xm[0] + q);
}

// x += alpha p, r -= alpha w; |r|^2, (r_new, y_old); max|r| into xm[1]; clears
// xm[0]; the last block books the iteration (convergence per right-hand side)
__global__ void k_l1_update(float2* x, float2* r, const float2* __restrict__ p, const float2* __restrict__ w,
                            const float2* __restrict__ y, size_t ne, int R, CtlL2* ctl, int par, int maxiter,
                            Reduction red) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < RMAX) ctl->xm[0][t] = 0u;
  double v[2 * RMAX];
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < 2 * RMAX; ++q) v[q] = 0.0;
#pragma unroll
  for (int q = 0; q < RMAX; ++q) m[q] = 0.f;
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const size_t o = t * R + q;
        float2 rv = r[o];
        // (p, A p) <= 0 (a rounded operator that is not positive definite at the
        // bottom of its spectrum) ends the right-hand side's iteration unchanged
        if (!ctl->done[q] && ctl->pAp[q] > 0.0) {
          const double pap = ctl->pAp[q];
          const float al = (float)(ctl->ry[par][q] / pap);
          const float2 pv = p[o], wv = w[o];
          float2 xv = x[o];
          xv.x += al * pv.x;
          xv.y += al * pv.y;
          rv.x -= al * wv.x;
          rv.y -= al * wv.y;
          x[o] = xv;
          r[o] = rv;
        }
        const float2 yv = y[o];
        v[q] = (double)rv.x * rv.x + (double)rv.y * rv.y;
        v[RMAX + q] = (double)rv.x * yv.x + (double)rv.y * yv.y;
        m[q] = fmaxf(fabsf(rv.x), fabsf(rv.y));
      }
#pragma unroll
  for (int q = 0; q < RMAX; ++q)
    if (q < R) warp_max_to(m[q], ctl->xm[1] + q);
  if (grid_reduce<2 * RMAX>(v, red, R) && threadIdx.x == 0) {
    const int it = ctl->iter + 1;
    ctl->iter = it;
    int all = 1;
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const double rn = ctl->rr[q];
        if (!ctl->done[q] && (rn <= ctl->stop[q] || it >= maxiter || !(rn == rn) || !(ctl->pAp[q] > 0.0))) {
          ctl->done[q] = 1;
          if (!(rn <= ctl->stop[q]) && it < maxiter) ctl->broke = 1;
        }
      }
      all &= ctl->done[q];
    }
    ctl->all_done = all;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void level2_init(Ctx& c, Coarse& A, const Subspace& s, const int block[4], int nvec) {
  HDCG_REQUIRE(nvec >= 1 && nvec <= L2_MAXV, HDCG_ERR_ARG, "level-2 nvec must be 1..64");
  HDCG_REQUIRE(A.vec_prec() == HDCG_F32, HDCG_ERR_ARG,
               "the blocked second coarsening needs an FP32 or FP16 little Dirac operator");
  for (int mu = 0; mu < 4; ++mu)
    HDCG_REQUIRE(block[mu] >= 1 && s.cdims[mu] % block[mu] == 0, HDCG_ERR_ARG,
                 "level-2 block extents must divide the coarse lattice extents");
  if (!A.l2) A.l2 = new Level2();
  Level2& L = *A.l2;
  L.have_A2 = false;
  L.graph.reset();
  L.Vc1 = s.Vc;
  L.n1 = s.nvec;
  L.nvec = nvec;
  L.spb = 1;
  L.Vc2 = 1;
  for (int mu = 0; mu < 4; ++mu) {
    L.block[mu] = block[mu];
    L.cdims[mu] = s.cdims[mu] / block[mu];
    L.spb *= block[mu];
    L.Vc2 *= L.cdims[mu];
  }
  HDCG_REQUIRE((size_t)nvec * L.Vc2 <= 65536, HDCG_ERR_ARG,
               "level-2 operator too large for its dense inverse (Vc2 * Nvec2 <= 65536)");
  std::vector<int> blk(L.Vc1), sites(L.Vc2 * L.spb), fill(L.Vc2, 0), coords(L.Vc2 * 4), nb(L.Vc2 * 81);
  for (size_t a = 0; a < L.Vc1; ++a) {
    size_t r = a, b = 0, mul = 1;
    for (int mu = 0; mu < 4; ++mu) {
      const int x = (int)(r % s.cdims[mu]);
      r /= s.cdims[mu];
      b += (size_t)(x / block[mu]) * mul;
      mul *= L.cdims[mu];
    }
    blk[a] = (int)b;
    sites[b * L.spb + fill[b]++] = (int)a;
  }
  for (size_t b = 0; b < L.Vc2; ++b) {
    size_t r = b;
    for (int mu = 0; mu < 4; ++mu) {
      coords[b * 4 + mu] = (int)(r % L.cdims[mu]);
      r /= L.cdims[mu];
    }
    for (int l = 0; l < 81; ++l) {
      int q = l;
      size_t idx = 0, mul = 1;
      for (int mu = 0; mu < 4; ++mu) {
        const int d = q % 3 - 1;
        q /= 3;
        const int y = ((coords[b * 4 + mu] + d) % L.cdims[mu] + L.cdims[mu]) % L.cdims[mu];
        idx += y * mul;
        mul *= L.cdims[mu];
      }
      nb[b * 81 + l] = (int)idx;
    }
  }
  L.blk_of_site.ensure(blk.size() * sizeof(int));
  L.sites.ensure(sites.size() * sizeof(int));
  L.coords.ensure(coords.size() * sizeof(int));
  L.cnbr2.ensure(nb.size() * sizeof(int));
  HDCG_CUDA(cudaMemcpy(L.blk_of_site.p, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice));
  HDCG_CUDA(cudaMemcpy(L.sites.p, sites.data(), sites.size() * sizeof(int), cudaMemcpyHostToDevice));
  HDCG_CUDA(cudaMemcpy(L.coords.p, coords.data(), coords.size() * sizeof(int), cudaMemcpyHostToDevice));
  HDCG_CUDA(cudaMemcpy(L.cnbr2.p, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
  L.phi.ensure((size_t)nvec * L.Vc1 * L.n1 * sizeof(float2));
}

// offsets stored on a lattice of extents d (bit l of the mask)
static std::vector<unsigned> keep_mask(const int d[4]) {
  std::vector<unsigned> m(3, 0u);
  for (int l = 0; l < 81; ++l) {
    int q = l;
    bool ok = true;
    for (int mu = 0; mu < 4; ++mu) {
      ok = ok && kept(q % 3 - 1, d[mu]);
      q /= 3;
    }
    if (ok) m[l >> 5] |= 1u << (l & 31);
  }
  return m;
}

void level2_orthonormalise(Ctx& c, Level2& L) {
  const int n = L.nvec;
  const size_t ne = L.Vc1 * L.n1;
  DevMem G, T, fail;
  G.ensure(L.Vc2 * n * n * sizeof(double2));
  T.ensure(L.Vc2 * n * n * sizeof(double2));
  fail.ensure(sizeof(int));
  HDCG_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), c.stream));
  const size_t sm = (size_t)n * L.n1 * sizeof(float2);
  smem_limit((const void*)k_l2_gram, sm);
  for (int round = 0; round < 2; ++round) {
    k_l2_gram<<<(unsigned)L.Vc2, 256, sm, c.stream>>>(L.phi.as<float2>(), ne, n, L.n1, L.sites.as<int>(), L.spb,
                                                       G.as<double2>());
    k_cholinv<<<(unsigned)((L.Vc2 + 63) / 64), 64, 0, c.stream>>>(G.as<double2>(), T.as<double2>(), n, L.Vc2,
                                                                  fail.as<int>());
    k_l2_transform<<<nblocks(ne), 256, 0, c.stream>>>(L.phi.as<float2>(), ne, n, L.n1, L.blk_of_site.as<int>(),
                                                       T.as<double2>());
    HDCG_CUDA(cudaGetLastError());
    c.launches += 3;
  }
  int h_fail = 0;
  HDCG_CUDA(cudaMemcpyAsync(&h_fail, fail.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  HDCG_REQUIRE(!h_fail, HDCG_ERR_BREAKDOWN,
               "level-2 block Gram matrix not positive definite (rank-deficient level-2 subspace)");
}

// [e][r] <-> [k][e] for a chunk of the level-2 vectors
__global__ void k_l2_gather(const float2* __restrict__ Z, size_t ne, int i0, int R, float2* X) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  X[t] = Z[(size_t)(i0 + (int)(t % R)) * ne + t / R];
}
__global__ void k_l2_scatter(const float2* __restrict__ X, size_t ne, int i0, int R, float2* Z) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  Z[(size_t)(i0 + (int)(t % R)) * ne + t / R] = X[t];
}

void level2_build_subspace(Ctx& c, Coarse& A, const Subspace& s, const hdcg_subspace_params& p) {
  level2_init(c, A, s, p.block, p.nvec);
  Level2& L = *A.l2;
  const size_t ne = L.Vc1 * L.n1;
  coarse_noise(c, L.phi.as<float2>(), (size_t)L.nvec * ne, p.seed);
  DevMem X, Y;
  X.ensure(ne * RMAX * sizeof(float2));
  Y.ensure(ne * RMAX * sizeof(float2));
  for (int step = 0; step < p.inv_steps; ++step) {
    for (int i0 = 0; i0 < L.nvec; i0 += RMAX) {
      const int R = std::min(RMAX, L.nvec - i0);
      k_l2_gather<<<nblocks(ne * R), 256, 0, c.stream>>>(L.phi.as<float2>(), ne, i0, R, X.as<float2>());
      ++c.launches;
      coarse_cg_multi(c, A, R, X.p, Y.p, p.inv_tol, p.inv_maxiter, p.inv_shift, false);
      k_l2_scatter<<<nblocks(ne * R), 256, 0, c.stream>>>(Y.as<float2>(), ne, i0, R, L.phi.as<float2>());
      ++c.launches;
      HDCG_CUDA(cudaGetLastError());
    }
    level2_orthonormalise(c, L);
  }
  if (p.inv_steps <= 0) level2_orthonormalise(c, L);
}

__global__ void k_l2_from_canon(const double2* __restrict__ in, float2* out, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = make_float2((float)in[t].x, (float)in[t].y);
}
__global__ void k_l2_to_canon(const float2* __restrict__ in, double2* out, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = make_double2(in[t].x, in[t].y);
}

void level2_set_subspace(Ctx& c, Coarse& A, const Subspace& s, const int block[4], int nvec, const void* phi,
                         int on_device, int already_orthonormal) {
  level2_init(c, A, s, block, nvec);
  Level2& L = *A.l2;
  const size_t n = (size_t)nvec * L.Vc1 * L.n1;
  DevMem tmp;
  const void* src = phi;
  if (!on_device) {
    tmp.ensure(n * sizeof(double2));
    HDCG_CUDA(cudaMemcpyAsync(tmp.p, phi, n * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    src = tmp.p;
  }
  k_l2_from_canon<<<nblocks(n), 256, 0, c.stream>>>((const double2*)src, L.phi.as<float2>(), n);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  if (!already_orthonormal) level2_orthonormalise(c, L);
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void level2_get_subspace(Ctx& c, const Coarse& A, void* host) {
  HDCG_REQUIRE(A.l2, HDCG_ERR_STATE, "no level-2 subspace");
  const Level2& L = *A.l2;
  const size_t n = (size_t)L.nvec * L.Vc1 * L.n1;
  DevMem tmp;
  tmp.ensure(n * sizeof(double2));
  k_l2_to_canon<<<nblocks(n), 256, 0, c.stream>>>(L.phi.as<float2>(), tmp.as<double2>(), n);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  HDCG_CUDA(cudaMemcpyAsync(host, tmp.p, n * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void level2_assemble(Ctx& c, Coarse& A, int inv_prec) {
  HDCG_REQUIRE(A.l2, HDCG_ERR_STATE, "no level-2 subspace");
  HDCG_REQUIRE(inv_prec == HDCG_F32 || inv_prec == HDCG_F64, HDCG_ERR_ARG,
               "the level-2 inverse is stored in F32 or F64");
  Level2& L = *A.l2;
  HDCG_REQUIRE(L.Vc1 == A.Vc && L.n1 == A.nvec, HDCG_ERR_STATE, "level-2 subspace does not match the operator");
  L.have_A2 = false;
  L.graph.reset();
  const int n = L.nvec, n1 = L.n1;
  const size_t ne = L.Vc1 * n1;
  // the most accurate copy of A: FP32 for an FP16 operator, A itself otherwise
  const void* Asrc = A.prec == HDCG_F16 ? A.Aacc.p : A.A.p;
  HDCG_REQUIRE(Asrc != nullptr, HDCG_ERR_STATE, "no FP32 copy of the FP16 little Dirac operator");
  L.A2.ensure(L.Vc2 * 81 * n * n * sizeof(double2));
  HDCG_CUDA(cudaMemsetAsync(L.A2.p, 0, L.Vc2 * 81 * n * n * sizeof(double2), c.stream));
  DevMem mask1, mask2, err;
  const std::vector<unsigned> m1 = keep_mask(reinterpret_cast<const int*>(c.sub->cdims));
  const std::vector<unsigned> m2 = keep_mask(L.cdims);
  mask1.ensure(3 * sizeof(unsigned));
  mask2.ensure(3 * sizeof(unsigned));
  err.ensure(sizeof(int));
  HDCG_CUDA(cudaMemcpyAsync(mask1.p, m1.data(), 3 * sizeof(unsigned), cudaMemcpyHostToDevice, c.stream));
  HDCG_CUDA(cudaMemcpyAsync(mask2.p, m2.data(), 3 * sizeof(unsigned), cudaMemcpyHostToDevice, c.stream));
  HDCG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream));
  const size_t sm = (size_t)(n1 * n1 + n1 * n) * sizeof(double2) + (size_t)2 * n * n1 * sizeof(float2);
  const int4 L2d = make_int4(L.cdims[0], L.cdims[1], L.cdims[2], L.cdims[3]);
  if (A.prec == HDCG_F64) {
    smem_limit((const void*)k_l2_galerkin<double2>, sm);
    k_l2_galerkin<double2><<<(unsigned)L.Vc1, 256, sm, c.stream>>>(
        (const double2*)Asrc, A.cnbr.as<int>(), n1, mask1.as<unsigned>(), L.phi.as<float2>(), ne, n,
        L.blk_of_site.as<int>(), L.coords.as<int>(), L2d, L.A2.as<double2>(), err.as<int>());
  } else {
    smem_limit((const void*)k_l2_galerkin<float2>, sm);
    k_l2_galerkin<float2><<<(unsigned)L.Vc1, 256, sm, c.stream>>>(
        (const float2*)Asrc, A.cnbr.as<int>(), n1, mask1.as<unsigned>(), L.phi.as<float2>(), ne, n,
        L.blk_of_site.as<int>(), L.coords.as<int>(), L2d, L.A2.as<double2>(), err.as<int>());
  }
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  // dense inverse of A2 (Jacobi-scaled)
  const size_t N = L.Vc2 * n;
  DevMem s, Pbuf;
  s.ensure(N * sizeof(double));
  Pbuf.ensure(GJB * GJB * sizeof(double2));
  k_l2_scale<<<nblocks(N), 256, 0, c.stream>>>(L.A2.as<double2>(), n, L.Vc2, s.as<double>(), err.as<int>());
  const size_t esz = inv_prec == HDCG_F64 ? sizeof(double2) : sizeof(float2);
  L.Ainv.release();
  L.Ainv.ensure(N * N * esz);
  L.inv_prec = inv_prec;
  HDCG_CUDA(cudaMemsetAsync(L.Ainv.p, 0, N * N * esz, c.stream));
  const size_t tot = L.Vc2 * 81 * n * n;
  if (inv_prec == HDCG_F64) {
    k_l2_dense<double2><<<nblocks(tot), 256, 0, c.stream>>>(L.A2.as<double2>(), L.cnbr2.as<int>(),
                                                             mask2.as<unsigned>(), n, L.Vc2, s.as<double>(),
                                                             L.Ainv.as<double2>());
    gj_inverse<double2>(c, L.Ainv.as<double2>(), N, Pbuf.as<double2>(), err.as<int>());
    k_l2_unscale<double2><<<nblocks(N * N), 256, 0, c.stream>>>(L.Ainv.as<double2>(), N, s.as<double>());
  } else {
    k_l2_dense<float2><<<nblocks(tot), 256, 0, c.stream>>>(L.A2.as<double2>(), L.cnbr2.as<int>(),
                                                            mask2.as<unsigned>(), n, L.Vc2, s.as<double>(),
                                                            L.Ainv.as<float2>());
    gj_inverse<float2>(c, L.Ainv.as<float2>(), N, Pbuf.as<double2>(), err.as<int>());
    k_l2_unscale<float2><<<nblocks(N * N), 256, 0, c.stream>>>(L.Ainv.as<float2>(), N, s.as<double>());
  }
  HDCG_CUDA(cudaGetLastError());
  c.launches += 3;
  int h_err = 0;
  HDCG_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  HDCG_REQUIRE(h_err == 0, HDCG_ERR_BREAKDOWN,
               h_err == 1 ? "level-2 operator: non-positive diagonal or a coupling beyond one block"
                          : "level-2 operator: zero or non-finite pivot in its inverse");
  L.have_A2 = true;
}

void level2_export(Ctx& c, const Coarse& A, void* host) {
  HDCG_REQUIRE(A.l2 && A.l2->have_A2, HDCG_ERR_STATE, "no level-2 operator");
  const Level2& L = *A.l2;
  HDCG_CUDA(cudaMemcpyAsync(host, L.A2.p, L.Vc2 * 81 * L.nvec * L.nvec * sizeof(double2), cudaMemcpyDeviceToHost,
                            c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// R2 / P2 / Q2 building blocks on [e][r] FP32 vectors
static void l2_restrict(Ctx& c, const Level2& L, const float2* x, const float2* xs, int R, float2* c2,
                        const int* skip) {
  const size_t sm = (size_t)(L.n1 * R + L.nvec * L.n1) * sizeof(float2);
  smem_limit((const void*)k_l2_restrict, sm);
  k_l2_restrict<<<(unsigned)L.Vc2, 256, sm, c.stream>>>(L.phi.as<float2>(), L.Vc1 * L.n1, L.nvec, L.n1,
                                                        L.sites.as<int>(), L.spb, x, xs, R, c2, skip);
  ++c.launches;
}
static void l2_prolong(Ctx& c, const Level2& L, const float2* c2, int R, const float2* add, float2* y,
                       const int* skip, double* dot, const float2* dv = nullptr) {
  const size_t ne = L.Vc1 * L.n1;
  const unsigned g = nblocks(ne);
  const Reduction red = dot ? make_reduction(c, g, RMAX, dot, 0) : Reduction{};
  k_l2_prolong<<<g, 256, 0, c.stream>>>(L.phi.as<float2>(), ne, L.nvec, L.n1, L.blk_of_site.as<int>(), c2, R, add, y,
                                        skip, red, dot ? 1 : 0, dv ? dv : add);
  ++c.launches;
}
static void l2_dense_solve(Ctx& c, const Level2& L, const float2* t, int R, float2* u, const int* skip) {
  const size_t N = L.Vc2 * L.nvec;
  if (L.inv_prec == HDCG_F64)
    k_dense_apply<double2><<<(unsigned)((N + 7) / 8), 256, 0, c.stream>>>(L.Ainv.as<double2>(), N, t, R, u, skip);
  else
    k_dense_apply<float2><<<(unsigned)((N + 7) / 8), 256, 0, c.stream>>>(L.Ainv.as<float2>(), N, t, R, u, skip);
  ++c.launches;
}

void level2_restrict_canon(Ctx& c, const Coarse& A, int R, const void* x64, void* c64) {
  HDCG_REQUIRE(A.l2, HDCG_ERR_STATE, "no level-2 subspace");
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  const Level2& L = *A.l2;
  const size_t ne = L.Vc1 * L.n1, n2 = L.Vc2 * L.nvec;
  DevMem x, cc;
  x.ensure(ne * R * sizeof(float2));
  cc.ensure(n2 * R * sizeof(float2));
  coarse_canon_to_multi(c, x64, x.as<float2>(), ne, R);
  l2_restrict(c, L, x.as<float2>(), nullptr, R, cc.as<float2>(), nullptr);
  coarse_multi_to_canon(c, cc.as<float2>(), c64, n2, R);
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void level2_prolong_canon(Ctx& c, const Coarse& A, int R, const void* c64, void* x64) {
  HDCG_REQUIRE(A.l2, HDCG_ERR_STATE, "no level-2 subspace");
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  const Level2& L = *A.l2;
  const size_t ne = L.Vc1 * L.n1, n2 = L.Vc2 * L.nvec;
  DevMem x, cc;
  x.ensure(ne * R * sizeof(float2));
  cc.ensure(n2 * R * sizeof(float2));
  coarse_canon_to_multi(c, c64, cc.as<float2>(), n2, R);
  l2_prolong(c, L, cc.as<float2>(), R, nullptr, x.as<float2>(), nullptr, nullptr);
  coarse_multi_to_canon(c, x.as<float2>(), x64, ne, R);
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

bool level2_active(const Coarse& A) { return A.l2 && A.l2->have_A2 && A.vec_prec() == HDCG_F32; }

// A x for R right-hand sides (FP32 [e][r]); xm: per-rhs max|x| already computed
// on the device; dot (may be null) receives Re<x, A x>
static void l1_apply(Ctx& c, Coarse& A, int R, const float2* x, float2* y, const unsigned* xm, const int* skip,
                     double* dot) {
  coarse_tc_to_b(c, A, R, x, xm, skip);
  coarse_tc_apply(c, A, R, x, y, xm, skip, dot, 0.0);
}

// The level-1 solve A x = b to |r| <= tol |b| (zero start): A-DEF2 with Q2 = P2 A2^-1 R2.
int level1_solve(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter) {
  HDCG_REQUIRE(level2_active(A), HDCG_ERR_STATE, "no level-2 operator");
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  coarse_tc_prepare(c, A);
  Level2& L = *A.l2;
  const size_t ne = L.Vc1 * L.n1, nc = ne * R, n2 = L.Vc2 * L.nvec * R;
  L.work.ensure((5 * nc + 2 * n2) * sizeof(float2));
  L.ctl.ensure(sizeof(CtlL2));
  float2* r = L.work.as<float2>();
  float2* p = r + nc;
  float2* w = p + nc;
  float2* y = w + nc;
  float2* c2 = y + nc;
  float2* u2 = c2 + n2;
  float2* zb = u2 + n2;      // M r (with the Q_trunc preconditioner)
  const float2* b = (const float2*)rhs;
  float2* x = (float2*)sol;
  CtlL2* ctl = L.ctl.as<CtlL2>();
  const int* skip = &ctl->all_done;
  const unsigned ge = nblocks(ne);
  HDCG_CUDA(cudaMemsetAsync(ctl, 0, sizeof(CtlL2), c.stream));
  // x0 = Q2 b; r0 = b - A x0; |b|^2
  k_l1_norm<<<ge, 256, 0, c.stream>>>(b, ne, R, make_reduction(c, ge, RMAX, ctl->bb, 0));
  ++c.launches;
  l2_restrict(c, L, b, nullptr, R, c2, nullptr);
  l2_dense_solve(c, L, c2, R, u2, nullptr);
  l2_prolong(c, L, u2, R, nullptr, x, nullptr, nullptr);
  coarse_tc_max(c, x, ne, R, ctl->xm[0]);
  l1_apply(c, A, R, x, w, ctl->xm[0], nullptr, nullptr);
  HDCG_CUDA(cudaMemsetAsync(ctl->xm[1], 0, RMAX * sizeof(unsigned), c.stream));
  k_l1_residual<<<ge, 256, 0, c.stream>>>(b, w, r, ne, R, ctl->xm[1], make_reduction(c, ge, RMAX, ctl->rr, 0));
  k_l1_start<<<1, 1, 0, c.stream>>>(ctl, R, tol, maxiter);
  c.launches += 2;
  // y = M1 r = z + Q2 (r - A z) with z = M r (M = 1, or the Chebyshev
  // polynomial of Q_trunc), (r, y) into ry[par]; w is scratch for A z
  const bool smooth = A.qt.order > 0;
  auto M1 = [&](int par) {
    const float2* z = r;
    const unsigned* xz = ctl->xm[1];
    if (smooth) {
      qtrunc_precondition(c, A, R, r, zb, ctl->xm[2], skip);
      z = zb;
      xz = ctl->xm[2];
    }
    l1_apply(c, A, R, z, w, xz, skip, nullptr);
    l2_restrict(c, L, r, w, R, c2, skip);
    l2_dense_solve(c, L, c2, R, u2, skip);
    l2_prolong(c, L, u2, R, z, y, skip, ctl->ry[par], r);
  };
  M1(0);
  k_l1_p<<<ge, 256, 0, c.stream>>>(p, y, ne, R, ctl, 0, 1);
  ++c.launches;
  // the iteration of parity par: w = A p; x, r update; y' = M1 r; p = y' + beta p
  auto iteration = [&](int par) {
    l1_apply(c, A, R, p, w, ctl->xm[0], skip, ctl->pAp);
    // |r|^2 and (r_new, y_old) land in ctl->rr and ctl->ryo (adjacent)
    k_l1_update<<<ge, 256, 0, c.stream>>>(x, r, p, w, y, ne, R, ctl, par, maxiter,
                                          make_reduction(c, ge, 2 * RMAX, ctl->rr, 0));
    ++c.launches;
    M1(par ^ 1);
    k_l1_p<<<ge, 256, 0, c.stream>>>(p, y, ne, R, ctl, par, 0);
    ++c.launches;
  };
  const std::vector<uintptr_t> key = {(uintptr_t)L.work.p, (uintptr_t)L.ctl.p, (uintptr_t)sol, (uintptr_t)rhs,
                                      (uintptr_t)A.Atc.p, (uintptr_t)A.xtc.p, (uintptr_t)A.tcs.p,
                                      (uintptr_t)L.Ainv.p, (uintptr_t)c.red_partials.p, (uintptr_t)c.red_ticket.p,
                                      (uintptr_t)R, (uintptr_t)maxiter, (uintptr_t)A.qt.order,
                                      (uintptr_t)A.qt.work.p, (uintptr_t)A.qt.A9.p};
  int queued = 0;
  int batch = std::max(2, L.last_iters);
  CtlL2 h{};
  HDCG_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CtlL2), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  while (!h.all_done) {
    for (int bq = 0; bq < batch && queued < maxiter; bq += 2, queued += 2) {
      if (queued == 0) {
        iteration(0);
        iteration(1);
      } else {
        run_captured(c, L.graph, key, [&] {
          iteration(0);
          iteration(1);
        });
      }
    }
    HDCG_CUDA(cudaGetLastError());
    HDCG_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CtlL2), cudaMemcpyDeviceToHost, c.stream));
    coarse_tc_check(c, A);   // synchronises the stream
    if (h.all_done || queued >= maxiter) break;
    batch = 2;
  }
  L.last_iters = std::max(2, h.iter);
  L.last_broke = h.broke;
  return h.iter;
}

}  // namespace hdcg
