// Second-level (global) deflation of the little Dirac operator and the A-DEF1
// coarse solver that uses it (Sec. 5.2, "Little Dirac operator deflation" and
// "Truncated little Dirac operator as preconditioner"; Table algos).
//
// Setup: nd Gaussian start vectors Z (the subspace generator's splitmix64
// stream), inv_steps steps of Z <- (A + shift)^-1 Z by the batched coarse CG
// (16 vectors per launch), each followed by Cholesky QR twice (FP64 Gram on
// the GPU, Cholesky on the host); then the prediagonalisation of the third,
// dense level: G = Z^dag A Z = S diag(lam) S^dag (Jacobi on the host),
// Z <- Z S, and W = Z - A Z is stored next to Z.
//
// A-DEF1 (M = 1, M_2 = M_3 = 1, V_start = 0): with d = diag(lam)^-1 Z^dag r,
//   y = M_1 r = P_L r + Q r = r - (A Z) d + Z d = r + W d,
// so an iteration applies A once (to p) and streams Z (for Z^dag r) and W
// (for y).  beta is the flexible (Polak-Ribiere) one.  The preconditioner is
// not symmetric, so (r, y) is taken by its real part.
#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

#include "coarse.cuh"

namespace hdcg {

namespace {

using cplx = std::complex<double>;
constexpr int LDOP_MAX = 256;
constexpr int DCH = 64;   // e-chunks of the per-iteration block dot

// ---------------------------------------------------------------------------
// host dense linear algebra of the third level
// ---------------------------------------------------------------------------

// Cyclic Jacobi for a Hermitian matrix (row-major n x n): each rotation first
// makes the pivot a_pq real by a phase on column q, then zeroes it with a real
// plane rotation.  Returns eigenvalues ascending and the unitary V (columns =
// eigenvectors, row-major V[i * n + k]).
void herm_eig(int n, std::vector<cplx> a, std::vector<double>& w, std::vector<cplx>& V) {
  V.assign((size_t)n * n, cplx(0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto A = [&](int i, int j) -> cplx& { return a[(size_t)i * n + j]; };
  double total = 0;
  for (auto& v : a) total += std::norm(v);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += std::norm(A(i, j));
    if (off <= 1e-30 * total || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cplx b = A(p, q);
        const double ab = std::abs(b);
        if (ab == 0.0) continue;
        const cplx e = b / ab;
        const double al = A(p, p).real(), ga = A(q, q).real();
        const double tau = (ga - al) / (2 * ab);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        const double cs = 1 / std::sqrt(1 + t * t), sn = t * cs;
        // J = [[cs, sn], [-sn conj(e), cs conj(e)]]
        const cplx j00 = cs, j01 = sn, j10 = -sn * std::conj(e), j11 = cs * std::conj(e);
        for (int i = 0; i < n; ++i) {   // columns p, q: A <- A J
          const cplx x = A(i, p), y = A(i, q);
          A(i, p) = x * j00 + y * j10;
          A(i, q) = x * j01 + y * j11;
        }
        for (int i = 0; i < n; ++i) {   // rows p, q: A <- J^dag A
          const cplx x = A(p, i), y = A(q, i);
          A(p, i) = std::conj(j00) * x + std::conj(j10) * y;
          A(q, i) = std::conj(j01) * x + std::conj(j11) * y;
        }
        A(p, q) = A(q, p) = 0;
        for (int i = 0; i < n; ++i) {   // V <- V J
          const cplx x = V[(size_t)i * n + p], y = V[(size_t)i * n + q];
          V[(size_t)i * n + p] = x * j00 + y * j10;
          V[(size_t)i * n + q] = x * j01 + y * j11;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return A(x, x).real() < A(y, y).real(); });
  std::vector<cplx> Vs((size_t)n * n);
  w.resize(n);
  for (int k = 0; k < n; ++k) {
    w[k] = A(order[k], order[k]).real();
    for (int i = 0; i < n; ++i) Vs[(size_t)i * n + k] = V[(size_t)i * n + order[k]];
  }
  V.swap(Vs);
}

// G = L L^dag (lower L, in place); false if G is not numerically positive definite
bool cholesky(int n, std::vector<cplx>& G) {
  for (int j = 0; j < n; ++j) {
    double d = G[(size_t)j * n + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(G[(size_t)j * n + k]);
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    G[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      cplx s = G[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= G[(size_t)i * n + k] * std::conj(G[(size_t)j * n + k]);
      G[(size_t)i * n + j] = s / d;
    }
    for (int i = 0; i < j; ++i) G[(size_t)i * n + j] = 0;
  }
  return true;
}

// T = L^-dag (upper triangular), so that Z T has orthonormal columns when Z^dag Z = L L^dag
std::vector<cplx> chol_whitener(int n, const std::vector<cplx>& L) {
  std::vector<cplx> Li((size_t)n * n, cplx(0));   // L^-1, lower
  for (int c = 0; c < n; ++c) {
    Li[(size_t)c * n + c] = 1.0 / L[(size_t)c * n + c];
    for (int i = c + 1; i < n; ++i) {
      cplx s = 0;
      for (int k = c; k < i; ++k) s += L[(size_t)i * n + k] * Li[(size_t)k * n + c];
      Li[(size_t)i * n + c] = -s / L[(size_t)i * n + i];
    }
  }
  std::vector<cplx> T((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) T[(size_t)i * n + k] = std::conj(Li[(size_t)k * n + i]);
  return T;
}

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------

// X[e][r] = Z[i0 + r][e]  /  Z[i0 + r][e] = X[e][r]
__global__ void k_gather(const float2* __restrict__ Z, size_t ne, int i0, int R, float2* X) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  const size_t e = t / R;
  const int r = (int)(t % R);
  X[t] = Z[(size_t)(i0 + r) * ne + e];
}
__global__ void k_scatter(const float2* __restrict__ X, size_t ne, int i0, int R, float2* Z) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  const size_t e = t / R;
  const int r = (int)(t % R);
  Z[(size_t)(i0 + r) * ne + e] = X[t];
}

// Gram partials: part[z][i][j] = sum_{e in chunk z} conj(X[i][e]) Y[j][e] in FP64
__global__ void __launch_bounds__(256) k_gram(const float2* __restrict__ X, const float2* __restrict__ Y, size_t ne,
                                              int nd, size_t chunk, double2* part) {
  __shared__ float2 xs[16][65], ys[16][65];
  const int ti = blockIdx.x * 16, tj = blockIdx.y * 16;
  const size_t e0 = blockIdx.z * chunk, e1 = min(ne, e0 + chunk);
  const int ii = threadIdx.x / 16, jj = threadIdx.x % 16;
  double ar = 0, ai = 0;
  for (size_t eb = e0; eb < e1; eb += 64) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int v = q / 64, ee = q % 64;
      const size_t e = eb + ee;
      xs[v][ee] = (ti + v < nd && e < e1) ? X[(size_t)(ti + v) * ne + e] : make_float2(0.f, 0.f);
      ys[v][ee] = (tj + v < nd && e < e1) ? Y[(size_t)(tj + v) * ne + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int ee = 0; ee < 64; ++ee) {
      const float2 a = xs[ii][ee], b = ys[jj][ee];
      ar += (double)a.x * b.x + (double)a.y * b.y;
      ai += (double)a.x * b.y - (double)a.y * b.x;
    }
    __syncthreads();
  }
  if (ti + ii < nd && tj + jj < nd) part[((size_t)blockIdx.z * nd + ti + ii) * nd + tj + jj] = make_double2(ar, ai);
}
__global__ void k_gram_reduce(const double2* __restrict__ part, int nch, int nd, double2* G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nd * nd) return;
  double ar = 0, ai = 0;
  for (int z = 0; z < nch; ++z) {
    const double2 v = part[(size_t)z * nd * nd + t];
    ar += v.x;
    ai += v.y;
  }
  G[t] = make_double2(ar, ai);
}

// Zout[k][e] = sum_i Z[i][e] T[i][k]  (T complex nd x nd, FP32), 16 outputs k per thread
__global__ void __launch_bounds__(256) k_transform(const float2* __restrict__ Z, const float2* __restrict__ T,
                                                   size_t ne, int nd, float2* Zout) {
  extern __shared__ float2 ts[];   // [nd][16]
  const int k0 = blockIdx.y * 16;
  for (int q = threadIdx.x; q < nd * 16; q += blockDim.x) {
    const int i = q / 16, kk = q % 16;
    ts[q] = k0 + kk < nd ? T[(size_t)i * nd + k0 + kk] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  float ar[16], ai[16];
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) ar[kk] = ai[kk] = 0.f;
  for (int i = 0; i < nd; ++i) {
    const float2 z = Z[(size_t)i * ne + e];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float2 t = ts[i * 16 + kk];
      ar[kk] += z.x * t.x - z.y * t.y;
      ai[kk] += z.x * t.y + z.y * t.x;
    }
  }
#pragma unroll
  for (int kk = 0; kk < 16; ++kk)
    if (k0 + kk < nd) Zout[(size_t)(k0 + kk) * ne + e] = make_float2(ar[kk], ai[kk]);
}

__global__ void k_sub(const float2* __restrict__ a, const float2* __restrict__ b, size_t n, float2* out) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = make_float2(a[t].x - b[t].x, a[t].y - b[t].y);
}

// y[e][r] = sum of ngroups partials w[g][e][r]
__global__ void k_sum_parts(const float2* __restrict__ w, size_t nc, int ngroups, float2* y) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  float2 v = w[t];
  for (int g = 1; g < ngroups; ++g) {
    v.x += w[(size_t)g * nc + t].x;
    v.y += w[(size_t)g * nc + t].y;
  }
  y[t] = v;
}

// ---- A-DEF1 iteration kernels ---------------------------------------------------

struct CCtlD {
  double rr[RMAX];
  double pAp[RMAX];
  double dots[2][2 * RMAX];   // [parity]: (r, y_new)[RMAX], (r, y_old)[RMAX]
  double stop[RMAX];
  int done[RMAX];
  int iter;
  int all_done;
};

// block dot partials: part[z][i][r] = sum_{e in chunk z} conj(Z[i][e]) V[e][r]
__global__ void __launch_bounds__(256) k_defl_dot(const float2* __restrict__ Z, const float2* __restrict__ V,
                                                  size_t ne, int nd, int R, size_t chunk, double2* part,
                                                  const int* skip) {
  if (skip && *skip) return;
  __shared__ float2 zs[16][65];
  __shared__ float2 vs[64][RMAX + 1];
  const int ti = blockIdx.x * 16;
  const size_t e0 = blockIdx.y * chunk, e1 = min(ne, e0 + chunk);
  const int ii = threadIdx.x / 16, rr = threadIdx.x % 16;
  float ar = 0.f, ai = 0.f;
  for (size_t eb = e0; eb < e1; eb += 64) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int v = q / 64, ee = q % 64;
      const size_t e = eb + ee;
      zs[v][ee] = (ti + v < nd && e < e1) ? Z[(size_t)(ti + v) * ne + e] : make_float2(0.f, 0.f);
      const int ee2 = q / RMAX, r2 = q % RMAX;
      const size_t f = eb + ee2;
      vs[ee2][r2] = (r2 < R && f < e1) ? V[f * R + r2] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int ee = 0; ee < 64; ++ee) {
      const float2 a = zs[ii][ee], b = vs[ee][rr];
      ar += a.x * b.x + a.y * b.y;
      ai += a.x * b.y - a.y * b.x;
    }
    __syncthreads();
  }
  if (ti + ii < nd) part[((size_t)blockIdx.y * nd + ti + ii) * RMAX + rr] = make_double2(ar, ai);
}

// d[i][r] = (sum_z part[z][i][r]) / lam_i  (a dropped pair has lam_i = +inf: d = 0)
__global__ void k_defl_dot_reduce(const double2* __restrict__ part, int nch, int nd, const double* __restrict__ lam,
                                  float2* d, const int* skip) {
  if (skip && *skip) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nd * RMAX) return;
  double ar = 0, ai = 0;
  for (int z = 0; z < nch; ++z) {
    const double2 v = part[(size_t)z * nd * RMAX + t];
    ar += v.x;
    ai += v.y;
  }
  const double il = 1.0 / lam[t / RMAX];
  d[t] = make_float2((float)(ar * il), (float)(ai * il));
}

// y = r + W d for every right-hand side; dots (r, y_new), (r, y_old).  A block
// takes 32 coarse unknowns e (lanes) and splits the nd vectors over its 8 warps;
// the warps' partial sums meet in shared memory.
constexpr int YE = 32, YG = 8;
__global__ void __launch_bounds__(YE * YG) k_defl_y(const float2* __restrict__ W, const float2* __restrict__ d,
                                                   const float2* __restrict__ r, float2* y, size_t ne, int nd,
                                                   int R, const int* skip, Reduction red) {
  if (skip && *skip) return;
  extern __shared__ float2 sm[];
  float2* ds = sm;                        // [nd][RMAX]
  float2* part = sm + (size_t)nd * RMAX;  // [YG][YE][RMAX]
  for (int q = threadIdx.x; q < nd * RMAX; q += blockDim.x) ds[q] = d[q];
  __syncthreads();
  const int lane = threadIdx.x % YE, grp = threadIdx.x / YE;
  const size_t e = (size_t)blockIdx.x * YE + lane;
  float ar[RMAX], ai[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) ar[q] = ai[q] = 0.f;
  if (e < ne) {
#pragma unroll 4
    for (int i = grp; i < nd; i += YG) {
      const float2 w = W[(size_t)i * ne + e];
#pragma unroll
      for (int q = 0; q < RMAX; ++q) {
        if (q < R) {
          const float2 dv = ds[i * RMAX + q];
          ar[q] += w.x * dv.x - w.y * dv.y;
          ai[q] += w.x * dv.y + w.y * dv.x;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RMAX; ++q)
    if (q < R) part[((size_t)grp * YE + lane) * RMAX + q] = make_float2(ar[q], ai[q]);
  __syncthreads();
  double v[2 * RMAX];
#pragma unroll
  for (int q = 0; q < 2 * RMAX; ++q) v[q] = 0.0;
  for (int idx = threadIdx.x; idx < YE * R; idx += blockDim.x) {
    const int q = idx / YE, l = idx % YE;
    const size_t f = (size_t)blockIdx.x * YE + l;
    if (f >= ne) continue;
    float sr = 0.f, si = 0.f;
    for (int g = 0; g < YG; ++g) {
      const float2 pv = part[((size_t)g * YE + l) * RMAX + q];
      sr += pv.x;
      si += pv.y;
    }
    const size_t o = f * R + q;
    const float2 rv = r[o], yo = y[o];
    const float yr = rv.x + sr, yi = rv.y + si;
    y[o] = make_float2(yr, yi);
    const double dn = (double)rv.x * yr + (double)rv.y * yi;
    const double dd = (double)rv.x * yo.x + (double)rv.y * yo.y;
#pragma unroll
    for (int qq = 0; qq < RMAX; ++qq)
      if (qq == q) {
        v[qq] += dn;
        v[RMAX + qq] += dd;
      }
  }
  grid_reduce<2 * RMAX>(v, red, R);
}

__global__ void k_ad1_init(const float2* __restrict__ b, float2* x, float2* r, float2* y, size_t ne, int R,
                           Reduction red) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) v[q] = 0.0;
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const float2 bv = b[t * R + q];
        x[t * R + q] = make_float2(0.f, 0.f);
        y[t * R + q] = make_float2(0.f, 0.f);
        r[t * R + q] = bv;
        v[q] = (double)bv.x * bv.x + (double)bv.y * bv.y;
      }
  grid_reduce<RMAX>(v, red, R);
}

__global__ void k_ad1_start(CCtlD* ctl, int R, double tol, int maxiter) {
  int all = 1;
  for (int q = 0; q < RMAX; ++q) {
    ctl->stop[q] = q < R ? tol * tol * ctl->rr[q] : 0.0;
    ctl->done[q] = q < R ? ((ctl->rr[q] == 0.0 || maxiter <= 0) ? 1 : 0) : 1;
    all &= ctl->done[q];
  }
  ctl->iter = 0;
  ctl->all_done = all;
}

// x += alpha p, r -= alpha w (running right-hand sides), |r|^2 into ctl->rr; clears
// xmax; then the convergence bookkeeping of the iteration
__global__ void k_ad1_update(float2* x, float2* r, const float2* __restrict__ p, const float2* __restrict__ w,
                             int ngroups, size_t ne, int R, CCtlD* ctl, int par, unsigned* xmax, int maxiter,
                             Reduction red) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0 && xmax)
    for (int q = 0; q < RMAX; ++q) xmax[q] = 0u;
  const size_t nc = ne * R;
  double v[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) v[q] = 0.0;
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const size_t o = t * R + q;
        float2 rv = r[o];
        if (!ctl->done[q]) {
          const double pap = ctl->pAp[q];
          const float al = (float)(pap != 0.0 ? ctl->dots[par][q] / pap : 0.0);
          float2 wv = w[o];
          for (int g = 1; g < ngroups; ++g) {
            wv.x += w[(size_t)g * nc + o].x;
            wv.y += w[(size_t)g * nc + o].y;
          }
          const float2 pv = p[o];
          float2 xv = x[o];
          xv.x += al * pv.x;
          xv.y += al * pv.y;
          rv.x -= al * wv.x;
          rv.y -= al * wv.y;
          x[o] = xv;
          r[o] = rv;
        }
        v[q] = (double)rv.x * rv.x + (double)rv.y * rv.y;
      }
    }
  // the last block, after every block has updated its part, books the iteration
  if (grid_reduce<RMAX>(v, red, R) && threadIdx.x == 0) {
    const int it = ctl->iter + 1;
    ctl->iter = it;
    int all = 1;
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const double rn = ctl->rr[q];
        if (!ctl->done[q] && (rn <= ctl->stop[q] || it >= maxiter || !(rn == rn))) ctl->done[q] = 1;
      }
      all &= ctl->done[q];
    }
    ctl->all_done = all;
  }
}

// p = y + beta p (flexible beta; first: p = y) for running right-hand sides; max|p|
__global__ void k_ad1_p(float2* p, const float2* __restrict__ y, size_t ne, int R, const CCtlD* ctl, int par,
                        int first, unsigned* xmax) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) m[q] = 0.f;
  if (t < ne)
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const size_t o = t * R + q;
        float2 pv = p[o];
        if (!ctl->done[q]) {
          float beta = 0.f;
          if (!first) {
            const double ry_old = ctl->dots[par ^ 1][q];
            beta = (float)(ry_old != 0.0 ? (ctl->dots[par][q] - ctl->dots[par][RMAX + q]) / ry_old : 0.0);
          }
          const float2 yv = y[o];
          pv.x = yv.x + beta * pv.x;
          pv.y = yv.y + beta * pv.y;
          p[o] = pv;
        }
        m[q] = fmaxf(fabsf(pv.x), fabsf(pv.y));
      }
    }
  if (!xmax) return;
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    if (q >= R) break;
    float u = m[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u = fmaxf(u, __shfl_xor_sync(FULL_MASK, u, o));
    if ((threadIdx.x & 31) == 0 && u > 0.f) atomicMax(xmax + q, __float_as_uint(u));
  }
}

unsigned blocks(size_t n) { return (unsigned)((n + 255) / 256); }

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

// G = X^dag Y (nd x nd, FP64, row-major G[i * nd + j] = <X_i, Y_j>) on the host
std::vector<cplx> gram(Ctx& c, const float2* X, const float2* Y, size_t ne, int nd) {
  const int nch = (int)std::min<size_t>(64, std::max<size_t>(1, ne / 4096));
  const size_t chunk = ((ne + nch - 1) / nch + 63) / 64 * 64;
  DevMem part, G;
  part.ensure((size_t)nch * nd * nd * sizeof(double2));
  G.ensure((size_t)nd * nd * sizeof(double2));
  const dim3 grid((nd + 15) / 16, (nd + 15) / 16, nch);
  k_gram<<<grid, 256, 0, c.stream>>>(X, Y, ne, nd, chunk, part.as<double2>());
  k_gram_reduce<<<blocks((size_t)nd * nd), 256, 0, c.stream>>>(part.as<double2>(), nch, nd, G.as<double2>());
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2;
  std::vector<cplx> h((size_t)nd * nd);
  HDCG_CUDA(cudaMemcpyAsync(h.data(), G.p, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

// Z <- Z T on the device (T host, nd x nd row-major)
void transform(Ctx& c, float2* Z, size_t ne, int nd, const std::vector<cplx>& T, DevMem& tmp) {
  std::vector<float2> tf(T.size());
  for (size_t i = 0; i < T.size(); ++i) tf[i] = make_float2((float)T[i].real(), (float)T[i].imag());
  DevMem Td;
  Td.ensure(tf.size() * sizeof(float2));
  HDCG_CUDA(cudaMemcpyAsync(Td.p, tf.data(), tf.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
  tmp.ensure((size_t)nd * ne * sizeof(float2));
  const size_t sm = (size_t)nd * 16 * sizeof(float2);
  if (sm > 48 * 1024)
    HDCG_CUDA(cudaFuncSetAttribute(k_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const dim3 grid(blocks(ne), (nd + 15) / 16);
  k_transform<<<grid, 256, sm, c.stream>>>(Z, Td.as<float2>(), ne, nd, tmp.as<float2>());
  HDCG_CUDA(cudaMemcpyAsync(Z, tmp.p, (size_t)nd * ne * sizeof(float2), cudaMemcpyDeviceToDevice, c.stream));
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// Cholesky QR of the columns of Z, three passes.  Inverse iteration makes the
// vectors nearly parallel, so the first pass factors G + sigma I (a diagonal
// shift of 1e-6 of the mean diagonal, raised tenfold while the factorisation
// fails); the shifted pass leaves Z well enough conditioned for two plain ones.
void orthonormalise(Ctx& c, float2* Z, size_t ne, int nd, DevMem& tmp) {
  for (int pass = 0; pass < 3; ++pass) {
    std::vector<cplx> G = gram(c, Z, Z, ne, nd);
    double tr = 0;
    for (int i = 0; i < nd; ++i) {
      for (int j = 0; j < i; ++j) G[(size_t)i * nd + j] = std::conj(G[(size_t)j * nd + i]);
      tr += G[(size_t)i * nd + i].real();
    }
    double sigma = pass == 0 ? 1e-6 * tr / nd : 0.0;
    bool ok = false;
    for (int attempt = 0; attempt < 8 && !ok; ++attempt) {
      std::vector<cplx> L = G;
      for (int i = 0; i < nd; ++i) L[(size_t)i * nd + i] += sigma;
      if (cholesky(nd, L)) {
        transform(c, Z, ne, nd, chol_whitener(nd, L), tmp);
        ok = true;
      } else {
        sigma = sigma > 0 ? 10 * sigma : 1e-6 * tr / nd;
      }
    }
    HDCG_REQUIRE(ok, HDCG_ERR_BREAKDOWN, "little Dirac deflation: the vectors could not be orthonormalised");
  }
}

// mean of the real diagonal of A (one block, fixed summation order)
template <typename AT>
__global__ void k_mean_diag(const AT* __restrict__ A, size_t Vc, int n, double* out) {
  double v[1] = {0.0};
  for (size_t t = threadIdx.x; t < Vc * n; t += blockDim.x) {
    const size_t a = t / n;
    const int j = (int)(t % n);
    const AT e = A[((a * 81 + 40) * n + j) * n + j];   // offset l = 40 is delta = 0
    if constexpr (sizeof(AT) == 8) v[0] += (double)reinterpret_cast<const float2&>(e).x;
    else v[0] += (double)__low2float(reinterpret_cast<const __half2&>(e));
  }
  block_sum<1>(v);
  if (threadIdx.x == 0) *out = v[0] / (double)(Vc * n);
}

double mean_diag(Ctx& c, const Coarse& A) {
  DevMem d;
  d.ensure(sizeof(double));
  if (A.prec == HDCG_F32) k_mean_diag<float2><<<1, 256, 0, c.stream>>>(A.A.as<float2>(), A.Vc, A.nvec, d.as<double>());
  else k_mean_diag<__half2><<<1, 256, 0, c.stream>>>(A.A.as<__half2>(), A.Vc, A.nvec, d.as<double>());
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  double h = 0;
  HDCG_CUDA(cudaMemcpyAsync(&h, d.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

// Y = A X for R <= 16 FP32 vectors [e][r] (tensor cores for FP16 A)
void apply_batch(Ctx& c, Coarse& A, int R, const float2* X, float2* Y, DevMem& part, DevMem& dots) {
  const size_t ne = A.Vc * A.nvec;
  dots.ensure(RMAX * sizeof(double));
  if (coarse_tc_supported(A)) {
    coarse_tc_prepare(c, A);
    unsigned* xmax = A.tcs.as<TcState>()->xmax;
    coarse_tc_max(c, X, ne, R, xmax);
    coarse_tc_to_b(c, A, R, X, xmax, nullptr);
    coarse_tc_apply(c, A, R, X, Y, xmax, nullptr, nullptr, 0.0);
    coarse_tc_check(c, A);
    return;
  }
  part.ensure((size_t)4 * ne * R * sizeof(float2));
  const int ng = coarse_apply_partials(c, A, R, X, part.as<float2>(), nullptr, dots.as<double>());
  k_sum_parts<<<blocks(ne * R), 256, 0, c.stream>>>(part.as<float2>(), ne * R, ng, Y);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

}  // namespace

// host entry to the third level's dense Hermitian eigensolver (no device work)
void dense_heev(int n, const double* H, double* w, double* V) {
  std::vector<cplx> a((size_t)n * n);
  for (size_t i = 0; i < a.size(); ++i) a[i] = cplx(H[2 * i], H[2 * i + 1]);
  for (int i = 0; i < n; ++i)   // use the Hermitian part
    for (int j = 0; j < i; ++j) {
      const cplx h = 0.5 * (a[(size_t)i * n + j] + std::conj(a[(size_t)j * n + i]));
      a[(size_t)i * n + j] = h;
      a[(size_t)j * n + i] = std::conj(h);
    }
  for (int i = 0; i < n; ++i) a[(size_t)i * n + i] = a[(size_t)i * n + i].real();
  std::vector<double> ww;
  std::vector<cplx> vv;
  herm_eig(n, a, ww, vv);
  std::copy(ww.begin(), ww.end(), w);
  if (V)
    for (size_t i = 0; i < vv.size(); ++i) {
      V[2 * i] = vv[i].real();
      V[2 * i + 1] = vv[i].imag();
    }
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------

void ldop_build(Ctx& c, Coarse& A, const hdcg_ldop_params& prm) {
  HDCG_REQUIRE(prm.nvec >= 0 && prm.nvec <= LDOP_MAX, HDCG_ERR_ARG, "0..256 little Dirac deflation vectors");
  auto& D = A.defl;
  D.nd = 0;
  D.lam_h.clear();
  A.graph_ad1.reset();
  if (prm.nvec == 0) {
    D.Z.release();
    D.W.release();
    D.lam.release();
    return;
  }
  HDCG_REQUIRE(A.prec == HDCG_F32 || A.prec == HDCG_F16, HDCG_ERR_ARG,
               "little Dirac deflation needs an FP32 or FP16 coarse operator");
  HDCG_REQUIRE(prm.inv_steps >= 0 && prm.tol > 0 && prm.maxiter > 0, HDCG_ERR_ARG,
               "inv_steps >= 0, tol > 0, maxiter > 0");
  // a negative shift is relative: |shift| times the mean diagonal element of A
  const double shift = prm.shift >= 0 ? prm.shift : -prm.shift * mean_diag(c, A);
  const int nd = prm.nvec;
  const size_t ne = A.Vc * A.nvec;
  HDCG_REQUIRE((size_t)nd <= ne, HDCG_ERR_ARG, "more deflation vectors than coarse unknowns");
  D.Z.ensure((size_t)nd * ne * sizeof(float2));
  D.W.ensure((size_t)nd * ne * sizeof(float2));
  float2* Z = D.Z.as<float2>();
  float2* AZ = D.W.as<float2>();   // holds A Z until W = Z - A Z is formed
  coarse_noise(c, Z, (size_t)nd * ne, prm.seed);
  DevMem tmp, X, Y, part, dots;
  X.ensure(ne * RMAX * sizeof(float2));
  Y.ensure(ne * RMAX * sizeof(float2));
  for (int step = 0; step < prm.inv_steps; ++step) {
    for (int i0 = 0; i0 < nd; i0 += RMAX) {
      const int R = std::min(RMAX, nd - i0);
      k_gather<<<blocks(ne * R), 256, 0, c.stream>>>(Z, ne, i0, R, X.as<float2>());
      c.launches += 1;
      coarse_cg_multi(c, A, R, X.p, Y.p, prm.tol, prm.maxiter, shift, false);
      k_scatter<<<blocks(ne * R), 256, 0, c.stream>>>(Y.as<float2>(), ne, i0, R, Z);
      c.launches += 1;
      HDCG_CUDA(cudaGetLastError());
    }
    orthonormalise(c, Z, ne, nd, tmp);
  }
  if (prm.inv_steps == 0) orthonormalise(c, Z, ne, nd, tmp);
  // Rayleigh-Ritz: G = Z^dag A Z = S diag(lam) S^dag
  for (int i0 = 0; i0 < nd; i0 += RMAX) {
    const int R = std::min(RMAX, nd - i0);
    k_gather<<<blocks(ne * R), 256, 0, c.stream>>>(Z, ne, i0, R, X.as<float2>());
    apply_batch(c, A, R, X.as<float2>(), Y.as<float2>(), part, dots);
    k_scatter<<<blocks(ne * R), 256, 0, c.stream>>>(Y.as<float2>(), ne, i0, R, AZ);
    c.launches += 2;
    HDCG_CUDA(cudaGetLastError());
  }
  std::vector<cplx> G = gram(c, Z, AZ, ne, nd);
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j <= i; ++j) {
      const cplx h = 0.5 * (G[(size_t)i * nd + j] + std::conj(G[(size_t)j * nd + i]));
      G[(size_t)i * nd + j] = h;
      G[(size_t)j * nd + i] = std::conj(h);
    }
  std::vector<double> lam;
  std::vector<cplx> S;
  herm_eig(nd, G, lam, S);
  // At light masses lam_min / lam_max of A (~1e-6 for m = 0.002 on 24^3 x 48) is
  // comparable to the rounding of an FP16 operator, and even to the error of an
  // FP32 Fourier assembly, so the computed operator need not be positive definite
  // at the very bottom.  Ritz pairs with lam <= 1e-7 lam_max are dropped from Q
  // (stored as lam = +inf, so d = Z^dag r / lam = 0 for them) rather than inverted.
  HDCG_REQUIRE(lam.back() > 0, HDCG_ERR_BREAKDOWN, "little Dirac deflation: no positive Ritz value");
  D.dropped = 0;
  for (double& l : lam)
    if (!(l > 1e-7 * lam.back())) {
      l = std::numeric_limits<double>::infinity();
      ++D.dropped;
    }
  transform(c, Z, ne, nd, S, tmp);
  transform(c, AZ, ne, nd, S, tmp);
  k_sub<<<blocks((size_t)nd * ne), 256, 0, c.stream>>>(Z, AZ, (size_t)nd * ne, AZ);   // W = Z - A Z
  c.launches += 1;
  D.lam.ensure(nd * sizeof(double));
  HDCG_CUDA(cudaMemcpyAsync(D.lam.p, lam.data(), nd * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  D.lam_h = lam;
  D.nd = nd;
}

void ldop_export(Ctx& c, const Coarse& A, double* lam_host, void* Z_host) {
  const auto& D = A.defl;
  HDCG_REQUIRE(D.nd > 0, HDCG_ERR_STATE, "no little Dirac deflation space");
  if (lam_host) std::copy(D.lam_h.begin(), D.lam_h.end(), lam_host);
  if (Z_host) {
    const size_t n = (size_t)D.nd * A.Vc * A.nvec;
    std::vector<float2> h(n);
    HDCG_CUDA(cudaMemcpyAsync(h.data(), D.Z.p, n * sizeof(float2), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    double* o = static_cast<double*>(Z_host);
    for (size_t i = 0; i < n; ++i) {
      o[2 * i] = h[i].x;
      o[2 * i + 1] = h[i].y;
    }
  }
}

// ---------------------------------------------------------------------------
// A-DEF1 coarse solve for R right-hand sides (FP32 vectors [a][k][r])
// ---------------------------------------------------------------------------

int coarse_adef1(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter) {
  auto& D = A.defl;
  HDCG_REQUIRE(D.nd > 0, HDCG_ERR_STATE, "no little Dirac deflation space");
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  const bool tc = coarse_tc_supported(A) && (R > 1 || coarse_use_tc_single(c, A));
  if (tc) coarse_tc_prepare(c, A);
  const int nd = D.nd;
  const size_t ne = A.Vc * A.nvec, nc = ne * R;
  const int ngp = tc ? 1 : 3;
  A.work.ensure((3 + ngp) * nc * sizeof(float2));
  // control block, then the block-dot partials, then d = lam^-1 Z^dag r
  const size_t off = (sizeof(CCtlD) + 255) / 256 * 256;
  A.ctl.ensure(off + (size_t)DCH * nd * RMAX * sizeof(double2) + (size_t)nd * RMAX * sizeof(float2));
  float2* r = A.work.as<float2>();
  float2* p = r + nc;
  float2* y = p + nc;
  float2* w = y + nc;
  CCtlD* ctl = A.ctl.as<CCtlD>();
  double2* dpart = reinterpret_cast<double2*>(A.ctl.as<char>() + off);
  float2* dvec = reinterpret_cast<float2*>(dpart + (size_t)DCH * nd * RMAX);
  unsigned* xmax = tc ? A.tcs.as<TcState>()->xmax : nullptr;
  const int* skip = &ctl->all_done;
  const unsigned ge = blocks(ne);
  const size_t chunk = ((ne + DCH - 1) / DCH + 63) / 64 * 64;
  const int nch = (int)((ne + chunk - 1) / chunk);
  const dim3 gdot((nd + 15) / 16, nch);
  const size_t ysm = ((size_t)nd * RMAX + YG * YE * RMAX) * sizeof(float2);
  // dynamic plus the reduction's static shared memory can pass the 48 KB default
  HDCG_CUDA(cudaFuncSetAttribute(k_defl_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm));
  const unsigned gy = (unsigned)((ne + YE - 1) / YE);
  const float2* Z = D.Z.as<float2>();
  const float2* W = D.W.as<float2>();
  const double* lam = D.lam.as<double>();

  auto precondition = [&](int par, int first) {
    k_defl_dot<<<gdot, 256, 0, c.stream>>>(Z, r, ne, nd, R, chunk, dpart, skip);
    k_defl_dot_reduce<<<blocks((size_t)nd * RMAX), 256, 0, c.stream>>>(dpart, nch, nd, lam, dvec, skip);
    k_defl_y<<<gy, YE * YG, ysm, c.stream>>>(W, dvec, r, y, ne, nd, R, skip,
                                              make_reduction(c, gy, 2 * RMAX, &ctl->dots[par][0], 0));
    k_ad1_p<<<ge, 256, 0, c.stream>>>(p, y, ne, R, ctl, par, first, xmax);
    c.launches += 4;
  };

  if (xmax) HDCG_CUDA(cudaMemsetAsync(xmax, 0, RMAX * sizeof(unsigned), c.stream));
  k_ad1_init<<<ge, 256, 0, c.stream>>>((const float2*)rhs, (float2*)sol, r, y, ne, R,
                                       make_reduction(c, ge, RMAX, &ctl->rr[0], 0));
  k_ad1_start<<<1, 1, 0, c.stream>>>(ctl, R, tol, maxiter);
  c.launches += 2;
  precondition(0, 1);
  // one iteration of parity par; iterations are queued in pairs (parities 0, 1),
  // the first pair directly and every later pair as a replayed CUDA graph
  auto iteration = [&](int par) {
    if (tc) {
      coarse_tc_to_b(c, A, R, p, xmax, skip);
      coarse_tc_apply(c, A, R, p, w, xmax, skip, &ctl->pAp[0], 0.0);
    } else {
      coarse_apply_partials(c, A, R, p, w, skip, &ctl->pAp[0]);
    }
    k_ad1_update<<<ge, 256, 0, c.stream>>>((float2*)sol, r, p, w, ngp, ne, R, ctl, par, xmax, maxiter,
                                           make_reduction(c, ge, RMAX, &ctl->rr[0], 0));
    c.launches += 1;
    precondition(par ^ 1, 0);
  };
  const std::vector<uintptr_t> key = {
      (uintptr_t)A.work.p, (uintptr_t)A.ctl.p, (uintptr_t)sol, (uintptr_t)D.Z.p, (uintptr_t)D.W.p,
      (uintptr_t)D.lam.p, (uintptr_t)(tc ? A.Atc.p : A.A.p), (uintptr_t)(tc ? A.xtc.p : nullptr),
      (uintptr_t)c.red_partials.p, (uintptr_t)c.red_ticket.p, (uintptr_t)A.tcs.p, (uintptr_t)R, (uintptr_t)nd,
      (uintptr_t)ne, (uintptr_t)tc, (uintptr_t)maxiter};
  int queued = 0;
  int batch = std::max(2, A.last_iters);
  CCtlD h{};
  while (true) {
    for (int bq = 0; bq < batch && queued < maxiter; bq += 2, queued += 2) {
      if (queued == 0) {
        iteration(0);
        iteration(1);
      } else {
        run_captured(c, A.graph_ad1, key, [&] {
          iteration(0);
          iteration(1);
        });
      }
    }
    HDCG_CUDA(cudaGetLastError());
    HDCG_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CCtlD), cudaMemcpyDeviceToHost, c.stream));
    if (tc) coarse_tc_check(c, A);
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    if (h.all_done || queued >= maxiter) break;
    batch = 2;
  }
  A.last_iters = std::max(1, h.iter);
  for (int q = 0; q < R; ++q)
    HDCG_REQUIRE(std::isfinite(h.rr[q]), HDCG_ERR_NONFINITE, "non-finite residual in the coarse A-DEF1 solve");
  return h.iter;
}

}  // namespace hdcg
