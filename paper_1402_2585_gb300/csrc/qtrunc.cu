// High-mode preconditioner of the little Dirac operator (Sec. 5.2, "Truncated
// little Dirac operator as preconditioner"; Table hierarchy: order 16 on
// [0.5, 45]).
//
// Q_trunc keeps the couplings of A within one block hop (the self block and
// the eight nearest neighbours, taxicab distance <= 1; pairs l, -l together,
// so it stays Hermitian), i.e. 9 of the 81 blocks.  M = p(Q_trunc + shift)
// with p the Chebyshev-acceleration polynomial of degree order - 1 on
// [lo, hi]:  1 - x p(x) = T_order((theta - x)/delta) / T_order(theta/delta),
// theta, delta the interval's midpoint and half-width.  p is positive below
// hi, so M is Hermitian positive definite when the spectrum of Q_trunc + shift
// lies below hi; hi defaults to 1.1 times a power-iteration estimate of its
// largest eigenvalue and lo to hi / 90 (the ratio of the paper's interval).
// Evaluated by the three-term recurrence of Chebyshev acceleration:
//   y_0 = 0, s_0 = r, d_0 = r / theta, rho_0 = delta / theta;
//   y_{k+1} = y_k + d_k, s_{k+1} = s_k - Q d_k,
//   rho_{k+1} = 1 / (2 theta / delta - rho_k),
//   d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) s_{k+1},
// order - 1 products with Q_trunc.  Vectors FP32 [e][r] (e = a Nvec + j).
#include <cmath>
#include <vector>

#include "coarse.cuh"

namespace hdcg {

namespace {

unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

// y[a][j][r] = sum_q sum_k A9[a][q][k][j] x[nb9[a][q]][k][r] + shift x[a][j][r],
// one warp per coarse site: lane l owns the outputs
// o = o0 + l + 32 u (u < U) of the current chunk, j = o / R, r = o % R.  Each
// row of a kept block (fixed q and k) is read coalesced across j, x[nb][k][r]
// is a broadcast within the warp, and no shared memory or barrier is needed.
template <int U>
__global__ void __launch_bounds__(256) k_qtrunc_apply_w(const float2* __restrict__ A9, const int* __restrict__ nb9,
                                                        int nq, int n, const float2* __restrict__ x, int R,
                                                        float shift, float2* y, const int* skip, size_t Vc) {
  if (skip && *skip) return;
  const size_t a = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (a >= Vc) return;
  const int lane = threadIdx.x & 31;
  const int nout = n * R;
  for (int o0 = 0; o0 < nout; o0 += 32 * U) {
    float ar[U], ai[U];
    int jo[U], ro[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int o = o0 + lane + 32 * u;
      live[u] = o < nout;
      jo[u] = live[u] ? o / R : 0;
      ro[u] = live[u] ? o % R : 0;
      ar[u] = 0.f;
      ai[u] = 0.f;
    }
    for (int q = 0; q < nq; ++q) {
      const size_t b = (size_t)__ldg(nb9 + a * 9 + q);
      const float2* blk = A9 + (a * 9 + q) * (size_t)n * n;
      const float2* xb = x + b * (size_t)nout;
#pragma unroll 4
      for (int k = 0; k < n; ++k) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (live[u]) {
            const float2 m = __ldg(blk + k * n + jo[u]);
            const float2 v = __ldg(xb + k * R + ro[u]);
            ar[u] += m.x * v.x - m.y * v.y;
            ai[u] += m.x * v.y + m.y * v.x;
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (live[u]) {
        const size_t o = a * (size_t)nout + o0 + lane + 32 * u;
        const float2 v = x[o];
        y[o] = make_float2(ar[u] + shift * v.x, ai[u] + shift * v.y);
      }
    }
  }
}

// d = r / theta, s = r, y = 0
__global__ void k_cheb_init(const float2* __restrict__ r, float2* d, float2* s, float2* y, size_t n, float itheta,
                            const int* skip) {
  if (skip && *skip) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float2 v = r[t];
  d[t] = make_float2(itheta * v.x, itheta * v.y);
  s[t] = v;
  y[t] = make_float2(0.f, 0.f);
}

// y += d; s -= q; d = c1 d + c2 s
__global__ void k_cheb_step(float2* y, float2* s, float2* d, const float2* __restrict__ q, size_t n, float c1, float c2,
                            const int* skip) {
  if (skip && *skip) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  float2 yv = y[t], sv = s[t], dv = d[t];
  const float2 qv = q[t];
  yv.x += dv.x;
  yv.y += dv.y;
  sv.x -= qv.x;
  sv.y -= qv.y;
  dv.x = c1 * dv.x + c2 * sv.x;
  dv.y = c1 * dv.y + c2 * sv.y;
  y[t] = yv;
  s[t] = sv;
  d[t] = dv;
}

// y += d; with xm != null, max(|Re y|, |Im y|) of each right-hand side into xm
// (cleared beforehand): the tensor-core operand scale of y
__global__ void k_cheb_last(float2* y, const float2* __restrict__ d, size_t ne, int R, unsigned* xm, const int* skip) {
  if (skip && *skip) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) m[q] = 0.f;
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const size_t o = t * R + q;
        float2 yv = y[o];
        const float2 dv = d[o];
        yv.x += dv.x;
        yv.y += dv.y;
        y[o] = yv;
        m[q] = fmaxf(fabsf(yv.x), fabsf(yv.y));
      }
  }
  if (!xm) return;
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    if (q >= R) break;
    float u = m[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u = fmaxf(u, __shfl_xor_sync(FULL_MASK, u, o));
    if ((threadIdx.x & 31) == 0 && u > 0.f) atomicMax(xm + q, __float_as_uint(u));
  }
}

template <typename AT>
__global__ void k_qtrunc_extract(const AT* __restrict__ A, const int* __restrict__ lsel, int nq, int n, size_t Vc,
                                 float2* A9) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)nq * n * n;
  if (t >= Vc * per) return;
  const size_t a = t / per;
  const int rem = (int)(t % per);
  const int q = rem / (n * n), e = rem % (n * n);
  const size_t src = ((a * 81 + lsel[q]) * n) * (size_t)n + e;
  if constexpr (sizeof(AT) == 16) {
    const double2 v = ((const double2*)A)[src];
    A9[(a * 9 + q) * (size_t)n * n + e] = make_float2((float)v.x, (float)v.y);
  } else {
    A9[(a * 9 + q) * (size_t)n * n + e] = ((const float2*)A)[src];
  }
}

__global__ void k_qtrunc_nb(const int* __restrict__ cnbr, const int* __restrict__ lsel, int nq, size_t Vc, int* nb9) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Vc * 9) return;
  const size_t a = t / 9;
  const int q = (int)(t % 9);
  nb9[t] = q < nq ? cnbr[a * 81 + lsel[q]] : 0;
}

// |v|^2 and Re<v, w> over n complex, one block (power iteration, setup only)
__global__ void k_pow_dots(const float2* __restrict__ v, const float2* __restrict__ w, size_t n, double* out) {
  double s[2] = {0.0, 0.0};
  for (size_t t = threadIdx.x; t < n; t += blockDim.x) {
    const float2 a = v[t], b = w[t];
    s[0] += (double)a.x * a.x + (double)a.y * a.y;
    s[1] += (double)a.x * b.x + (double)a.y * b.y;
  }
  block_sum<2>(s);
  if (threadIdx.x == 0) {
    out[0] = s[0];
    out[1] = s[1];
  }
}

// v = w / sqrt(nrm[0]) (nrm[0] = |w|^2)
__global__ void k_pow_norm(const float2* __restrict__ w, float2* v, size_t n, const double* nrm) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float f = (float)(1.0 / sqrt(nrm[0]));
  v[t] = make_float2(f * w[t].x, f * w[t].y);
}

}  // namespace

void qtrunc_apply(Ctx& c, const Coarse& A, int R, const float2* x, float2* y, double shift, const int* skip) {
  const QTrunc& Q = A.qt;
  const int nout = A.nvec * R;
  const unsigned grid = (unsigned)((A.Vc + 7) / 8);
  if (nout <= 32)
    k_qtrunc_apply_w<1><<<grid, 256, 0, c.stream>>>(Q.A9.as<float2>(), Q.nb9.as<int>(), Q.nq, A.nvec, x, R,
                                                   (float)shift, y, skip, A.Vc);
  else if (nout <= 64)
    k_qtrunc_apply_w<2><<<grid, 256, 0, c.stream>>>(Q.A9.as<float2>(), Q.nb9.as<int>(), Q.nq, A.nvec, x, R,
                                                   (float)shift, y, skip, A.Vc);
  else
    k_qtrunc_apply_w<4><<<grid, 256, 0, c.stream>>>(Q.A9.as<float2>(), Q.nb9.as<int>(), Q.nq, A.nvec, x, R,
                                                   (float)shift, y, skip, A.Vc);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// y = M r for R right-hand sides (FP32 [e][r]); xm (nullable, cleared here)
// receives the per-rhs max |y| for a following tensor-core apply
void qtrunc_precondition(Ctx& c, Coarse& A, int R, const float2* r, float2* y, unsigned* xm, const int* skip) {
  QTrunc& Q = A.qt;
  const size_t ne = A.Vc * A.nvec, nc = ne * R;
  Q.work.ensure(3 * nc * sizeof(float2));
  float2* s = Q.work.as<float2>();
  float2* d = s + nc;
  float2* t = d + nc;
  const double theta = 0.5 * (Q.hi + Q.lo), delta = 0.5 * (Q.hi - Q.lo);
  const unsigned g = nblk(nc);
  if (xm) HDCG_CUDA(cudaMemsetAsync(xm, 0, RMAX * sizeof(unsigned), c.stream));
  k_cheb_init<<<g, 256, 0, c.stream>>>(r, d, s, y, nc, (float)(1.0 / theta), skip);
  double rho = delta / theta;
  for (int k = 0; k + 1 < Q.order; ++k) {
    qtrunc_apply(c, A, R, d, t, Q.shift, skip);
    const double rn = 1.0 / (2.0 * theta / delta - rho);
    k_cheb_step<<<g, 256, 0, c.stream>>>(y, s, d, t, nc, (float)(rn * rho), (float)(2.0 * rn / delta), skip);
    rho = rn;
  }
  k_cheb_last<<<nblk(ne), 256, 0, c.stream>>>(y, d, ne, R, xm, skip);
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2 + std::max(0, Q.order - 1);
}

void qtrunc_setup(Ctx& c, Coarse& A, int order, double lo, double hi, double shift) {
  QTrunc& Q = A.qt;
  Q.order = 0;
  if (order <= 0) return;
  HDCG_REQUIRE(A.vec_prec() == HDCG_F32, HDCG_ERR_ARG, "the Q_trunc preconditioner needs an FP32 or FP16 operator");
  HDCG_REQUIRE(A.nvec <= 64, HDCG_ERR_ARG, "Nvec <= 64");
  // the stored offsets within one block hop
  int cd[4] = {0, 0, 0, 0};
  {
    // coarse extents from the neighbour table's reach: recover them from Vc's factorisation
    // through the subspace (the only owner of the geometry)
    const Subspace* s = c.sub;
    HDCG_REQUIRE(s, HDCG_ERR_STATE, "no subspace");
    for (int mu = 0; mu < 4; ++mu) cd[mu] = s->cdims[mu];
  }
  std::vector<int> lsel;
  for (int l = 0; l < 81; ++l) {
    int q = l, hops = 0;
    bool ok = true;
    for (int mu = 0; mu < 4; ++mu) {
      const int d = q % 3 - 1;
      q /= 3;
      hops += d != 0;
      const int L = cd[mu];
      ok = ok && (L >= 3 || (L == 2 ? d >= 0 : d == 0));
    }
    if (ok && hops <= 1) lsel.push_back(l);
  }
  Q.nq = (int)lsel.size();
  const int n = A.nvec;
  DevMem dl;
  dl.ensure(lsel.size() * sizeof(int));
  HDCG_CUDA(cudaMemcpyAsync(dl.p, lsel.data(), lsel.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  Q.A9.ensure(A.Vc * 9 * (size_t)n * n * sizeof(float2));
  Q.nb9.ensure(A.Vc * 9 * sizeof(int));
  const size_t tot = A.Vc * (size_t)Q.nq * n * n;
  const void* src = A.prec == HDCG_F16 ? A.Aacc.p : A.A.p;
  HDCG_REQUIRE(src, HDCG_ERR_STATE, "no FP32 copy of the FP16 little Dirac operator");
  if (A.prec == HDCG_F64)
    k_qtrunc_extract<double2><<<nblk(tot), 256, 0, c.stream>>>((const double2*)src, dl.as<int>(), Q.nq, n, A.Vc,
                                                               Q.A9.as<float2>());
  else
    k_qtrunc_extract<float2><<<nblk(tot), 256, 0, c.stream>>>((const float2*)src, dl.as<int>(), Q.nq, n, A.Vc,
                                                              Q.A9.as<float2>());
  k_qtrunc_nb<<<nblk(A.Vc * 9), 256, 0, c.stream>>>(A.cnbr.as<int>(), dl.as<int>(), Q.nq, A.Vc, Q.nb9.as<int>());
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2;
  Q.shift = shift;
  if (!(hi > 0)) {
    // largest eigenvalue of Q_trunc + shift: power iteration from a Gaussian
    // vector (the coarse noise stream, seed 0x5157), Rayleigh quotient
    const size_t ne = A.Vc * n;
    DevMem v, w, dots;
    v.ensure(ne * sizeof(float2));
    w.ensure(ne * sizeof(float2));
    dots.ensure(2 * sizeof(double));
    coarse_noise(c, v.as<float2>(), ne, 0x5157ull);
    double h[2] = {1.0, 0.0};
    for (int it = 0; it < 100; ++it) {
      qtrunc_apply(c, A, 1, v.as<float2>(), w.as<float2>(), shift, nullptr);
      k_pow_dots<<<1, 1024, 0, c.stream>>>(v.as<float2>(), w.as<float2>(), ne, dots.as<double>());
      k_pow_dots<<<1, 1024, 0, c.stream>>>(w.as<float2>(), w.as<float2>(), ne, dots.as<double>() + 0);
      k_pow_norm<<<nblk(ne), 256, 0, c.stream>>>(w.as<float2>(), v.as<float2>(), ne, dots.as<double>());
      c.launches += 4;
    }
    // Rayleigh quotient of the last normalised vector
    qtrunc_apply(c, A, 1, v.as<float2>(), w.as<float2>(), shift, nullptr);
    k_pow_dots<<<1, 1024, 0, c.stream>>>(v.as<float2>(), w.as<float2>(), ne, dots.as<double>());
    c.launches += 2;
    HDCG_CUDA(cudaMemcpyAsync(h, dots.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    HDCG_REQUIRE(h[0] > 0 && std::isfinite(h[1]), HDCG_ERR_NONFINITE, "Q_trunc power iteration failed");
    hi = 1.1 * h[1] / h[0];
  }
  if (!(lo > 0)) lo = hi * (lo < 0 ? -lo : 1.0 / 90.0);
  HDCG_REQUIRE(lo > 0 && hi > lo, HDCG_ERR_ARG, "the Chebyshev interval needs 0 < lo < hi");
  Q.lo = lo;
  Q.hi = hi;
  Q.order = order;
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// canonical [R][Vc][Nvec] complex double in and out (device): y = M x
void qtrunc_precondition_canon(Ctx& c, Coarse& A, int R, const void* x64, void* y64) {
  HDCG_REQUIRE(A.qt.order > 0, HDCG_ERR_STATE, "no coarse preconditioner");
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  const size_t ne = A.Vc * A.nvec;
  DevMem x, y;
  x.ensure(ne * R * sizeof(float2));
  y.ensure(ne * R * sizeof(float2));
  coarse_canon_to_multi(c, x64, x.as<float2>(), ne, R);
  qtrunc_precondition(c, A, R, x.as<float2>(), y.as<float2>(), nullptr, nullptr);
  coarse_multi_to_canon(c, y.as<float2>(), y64, ne, R);
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace hdcg
