// Fine operator of the HDCG library: the red-black preconditioned Shamir /
// Moebius domain-wall operator Mpc = M_oo - M_oe M_ee^-1 M_eo and
// H = Mpc^dag Mpc (Boyle, arXiv 1402.2585, Sec. 4), with
//   M_ee = M_oo = alpha + beta P_s,  M_eo = -Dh_eo K / 2,  K = b + c P_s,
//   alpha = b (4 - M5) + 1,  beta = c (4 - M5) - 1,
//   (P_s psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},  psi_{Ls} -> -m psi_0, psi_{-1} -> -m psi_{Ls-1}.
//
// H runs as four fused hop passes (each one launch):
//   A  (e <- o):  t   = K M_ee^-1 Dh_eo (K psi)
//   B  (o <- e):  chi = M_oo psi - Dh_oe t / 4                 [+ |chi|^2 in FP64]
//   C  (e <- o):  u   = M_ee^-dag K^dag Dh^dag_eo chi
//   D  (o <- e):  out = M_oo^dag chi - K^dag Dh^dag_oe u / 4   [+ optional lam * extra]
// Dh^dag is Dh with gamma_mu -> -gamma_mu.  One thread owns one 5D site; the
// Ls threads of a 4D site are consecutive lanes of one warp, so the
// s-direction operators (all polynomials in the twisted shift P_s, per
// chirality) run as warp shuffles: P_s^d is one shuffle per real, and
// M_ee^-1 = minv_norm * sum_{k<Ls} r^k P_s^k (r = -beta/alpha, P_s^Ls = -m)
// is evaluated by log2(Ls) doubling steps.  The gauge links of a 4D site are
// read once per CTA group and reused by its Ls lanes (Sec. 6.5: Ls-fold link reuse).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "context.h"

namespace hdcg {

struct HopArgs {
  const uint4* in;
  const uint4* in2;
  const uint4* extra;
  uint4* out;
  const void* links;
  const int* nbr;
  size_t n5;
  int Ls, lslog2;
  double b, c, alpha, beta, mass, minv_norm, rpow[6];
  double sD, lam;
  Reduction red;
  int do_red;
};

// ------------------------------------------------------------------------------
// link loads: 9 complex of one link into 18 reals
// ------------------------------------------------------------------------------
__device__ __forceinline__ void load_link(const double2* __restrict__ p, double* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double2 v = __ldg(p + i);
    u[2 * i] = v.x;
    u[2 * i + 1] = v.y;
  }
}
__device__ __forceinline__ void load_link(const float2* __restrict__ p, float* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    float2 v = __ldg(p + i);
    u[2 * i] = v.x;
    u[2 * i + 1] = v.y;
  }
}
__device__ __forceinline__ void load_link(const __half2* __restrict__ p, float* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    float2 v = __half22float2(__ldg(p + i));
    u[2 * i] = v.x;
    u[2 * i + 1] = v.y;
  }
}
__device__ __forceinline__ void load_link(const __nv_bfloat162* __restrict__ p, float* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    float2 v = __bfloat1622float2(__ldg(p + i));
    u[2 * i] = v.x;
    u[2 * i + 1] = v.y;
  }
}

// ------------------------------------------------------------------------------
// s-direction operators on one lane's 24 reals; spins 0,1 are chirality +
// (gamma5 = +1), spins 2,3 chirality -.  P_s acts on chirality + as the down
// shift (psi_{s-1}) and on chirality - as the up shift (psi_{s+1}); P_s^dag
// swaps them.  Wrapped values pick up -m.
// ------------------------------------------------------------------------------
template <typename R, bool DAG>
__device__ __forceinline__ void apply_Ppow(R* v, int d, int s, int Ls, R m) {
  const int up_src = (s + d) & (Ls - 1);
  const R up_f = (s + d >= Ls) ? -m : R(1);
  const int dn_src = (s - d) & (Ls - 1);
  const R dn_f = (s < d) ? -m : R(1);
  const int sp = DAG ? up_src : dn_src;
  const R fp = DAG ? up_f : dn_f;
  const int sm = DAG ? dn_src : up_src;
  const R fm = DAG ? dn_f : up_f;
#pragma unroll
  for (int i = 0; i < 12; ++i) v[i] = fp * __shfl_sync(FULL_MASK, v[i], sp, Ls);
#pragma unroll
  for (int i = 12; i < 24; ++i) v[i] = fm * __shfl_sync(FULL_MASK, v[i], sm, Ls);
}

// v <- a v + b P v
template <typename R, bool DAG>
__device__ __forceinline__ void apply_lin(R* v, R a, R b, int s, int Ls, R m) {
  R t[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) t[i] = v[i];
  apply_Ppow<R, DAG>(t, 1, s, Ls, m);
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] = a * v[i] + b * t[i];
}

// v <- M_ee^-1 v (DAG: M_ee^-dag) by doubling: A_{j+1} = A_j + r^{2^j} P^{2^j} A_j
template <typename R, bool DAG>
__device__ __forceinline__ void apply_minv(R* v, int s, const HopArgs& a) {
  const R m = (R)a.mass;
  for (int j = 0; j < a.lslog2; ++j) {
    R t[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) t[i] = v[i];
    apply_Ppow<R, DAG>(t, 1 << j, s, a.Ls, m);
    const R rp = (R)a.rpow[j];
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] += rp * t[i];
  }
  const R nrm = (R)a.minv_norm;
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] *= nrm;
}

// ------------------------------------------------------------------------------
// spin projection (1 - SG gamma_MU) in the chiral basis:
//   h = u - SG A_mu l,  result = (h, -SG B_mu h),  with A_mu, B_mu the 2x2
//   off-diagonal blocks of gamma_mu (A_mu B_mu = 1):
//   A_x l = (-i l1, -i l0), A_y l = (-l1, l0), A_z l = (-i l0, i l1), A_t l = (l0, l1)
//   B_x h = (i h1, i h0),   B_y h = (h1, -h0), B_z h = (i h0, -i h1), B_t h = (h0, h1)
// spinor reals index: (spin * 3 + colour) * 2 + {re, im}
// ------------------------------------------------------------------------------
template <int MU, int SG, typename R>
__device__ __forceinline__ void project(const R* p, R* h) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R u0r = p[(0 * 3 + c) * 2], u0i = p[(0 * 3 + c) * 2 + 1];
    const R u1r = p[(1 * 3 + c) * 2], u1i = p[(1 * 3 + c) * 2 + 1];
    const R l0r = p[(2 * 3 + c) * 2], l0i = p[(2 * 3 + c) * 2 + 1];
    const R l1r = p[(3 * 3 + c) * 2], l1i = p[(3 * 3 + c) * 2 + 1];
    R a0r, a0i, a1r, a1i;  // A_mu l
    if (MU == 0) { a0r = l1i; a0i = -l1r; a1r = l0i; a1i = -l0r; }
    else if (MU == 1) { a0r = -l1r; a0i = -l1i; a1r = l0r; a1i = l0i; }
    else if (MU == 2) { a0r = l0i; a0i = -l0r; a1r = -l1i; a1i = l1r; }
    else { a0r = l0r; a0i = l0i; a1r = l1r; a1i = l1i; }
    if (SG > 0) {
      h[(0 * 3 + c) * 2] = u0r - a0r; h[(0 * 3 + c) * 2 + 1] = u0i - a0i;
      h[(1 * 3 + c) * 2] = u1r - a1r; h[(1 * 3 + c) * 2 + 1] = u1i - a1i;
    } else {
      h[(0 * 3 + c) * 2] = u0r + a0r; h[(0 * 3 + c) * 2 + 1] = u0i + a0i;
      h[(1 * 3 + c) * 2] = u1r + a1r; h[(1 * 3 + c) * 2 + 1] = u1i + a1i;
    }
  }
}

// acc += (uh, -SG B_mu uh)
template <int MU, int SG, typename R>
__device__ __forceinline__ void reconstruct_add(const R* uh, R* acc) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R h0r = uh[(0 * 3 + c) * 2], h0i = uh[(0 * 3 + c) * 2 + 1];
    const R h1r = uh[(1 * 3 + c) * 2], h1i = uh[(1 * 3 + c) * 2 + 1];
    R b0r, b0i, b1r, b1i;  // B_mu h
    if (MU == 0) { b0r = -h1i; b0i = h1r; b1r = -h0i; b1i = h0r; }
    else if (MU == 1) { b0r = h1r; b0i = h1i; b1r = -h0r; b1i = -h0i; }
    else if (MU == 2) { b0r = -h0i; b0i = h0r; b1r = h1i; b1i = -h1r; }
    else { b0r = h0r; b0i = h0i; b1r = h1r; b1i = h1i; }
    acc[(0 * 3 + c) * 2] += h0r;
    acc[(0 * 3 + c) * 2 + 1] += h0i;
    acc[(1 * 3 + c) * 2] += h1r;
    acc[(1 * 3 + c) * 2 + 1] += h1i;
    if (SG > 0) {
      acc[(2 * 3 + c) * 2] -= b0r; acc[(2 * 3 + c) * 2 + 1] -= b0i;
      acc[(3 * 3 + c) * 2] -= b1r; acc[(3 * 3 + c) * 2 + 1] -= b1i;
    } else {
      acc[(2 * 3 + c) * 2] += b0r; acc[(2 * 3 + c) * 2 + 1] += b0i;
      acc[(3 * 3 + c) * 2] += b1r; acc[(3 * 3 + c) * 2 + 1] += b1i;
    }
  }
}

// uh[sp][a] = sum_b U[a][b] h[sp][b]
template <typename R>
__device__ __forceinline__ void su3_mul(const R* U, const R* h, R* uh) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R re = 0, im = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R ur = U[(a * 3 + b) * 2], ui = U[(a * 3 + b) * 2 + 1];
        const R hr = h[(sp * 3 + b) * 2], hi = h[(sp * 3 + b) * 2 + 1];
        re += ur * hr - ui * hi;
        im += ur * hi + ui * hr;
      }
      uh[(sp * 3 + a) * 2] = re;
      uh[(sp * 3 + a) * 2 + 1] = im;
    }
}

template <typename St> struct LinkOf;
template <> struct LinkOf<f64_t> { using T = double2; };
template <> struct LinkOf<f32_t> { using T = float2; };
template <> struct LinkOf<f16_t> { using T = __half2; };
template <> struct LinkOf<bf16_t> { using T = __nv_bfloat162; };
template <> struct LinkOf<bf16t_t> { using T = __nv_bfloat162; };

// both hops along direction MU: forward (x + mu, projector 1 - SF g) and
// backward (x - mu, projector 1 + SF g); the two neighbour spinors and links are
// loaded before either is used so that their loads overlap.
template <typename St, typename R, typename LT, int MU, int SF, bool KIN>
__device__ __forceinline__ void hop_pair(const HopArgs& a, const int* nbv, const LT* lk, int s, R* acc) {
  R pf[24], pb[24];
  load_spinor<St, R>(a.in, (size_t)nbv[MU] * a.Ls + s, a.n5, pf);
  load_spinor<St, R>(a.in, (size_t)nbv[MU + 4] * a.Ls + s, a.n5, pb);
  if (KIN) {
    const R m = (R)a.mass;
    apply_lin<R, false>(pf, (R)a.b, (R)a.c, s, a.Ls, m);
    apply_lin<R, false>(pb, (R)a.b, (R)a.c, s, a.Ls, m);
  }
  R h[12], uh[12], U[18];
  project<MU, SF>(pf, h);
  load_link(lk + MU * 9, U);
  su3_mul<R>(U, h, uh);
  reconstruct_add<MU, SF>(uh, acc);
  project<MU, -SF>(pb, h);
  load_link(lk + (MU + 4) * 9, U);
  su3_mul<R>(U, h, uh);
  reconstruct_add<MU, -SF>(uh, acc);
}

// ------------------------------------------------------------------------------
// one hop pass
// ------------------------------------------------------------------------------
template <typename St, int PASS, bool MOB>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs a) {
  using R = typename Store<St>::real;
  using LT = typename LinkOf<St>::T;
  constexpr bool DAG = (PASS == PASS_C || PASS == PASS_D);
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gtid < a.n5;
  const int s = threadIdx.x & (a.Ls - 1);
  const size_t x4 = active ? (gtid >> a.lslog2) : 0;
  const size_t site5 = x4 * a.Ls + s;
  const R m = (R)a.mass;

  R acc[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = 0;

  // all eight neighbour indices at once (32 bytes, shared by the Ls lanes of a site)
  const int4 nb0 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2);
  const int4 nb1 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2 + 1);
  const int nbv[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};
  const LT* lk = reinterpret_cast<const LT*>(a.links) + x4 * 72;
  // Dh: forward (1 - g), backward (1 + g); Dh^dag flips both.
  constexpr int SF = DAG ? -1 : 1;
  hop_pair<St, R, LT, 0, SF, PASS == PASS_A && MOB>(a, nbv, lk, s, acc);
  hop_pair<St, R, LT, 1, SF, PASS == PASS_A && MOB>(a, nbv, lk, s, acc);
  hop_pair<St, R, LT, 2, SF, PASS == PASS_A && MOB>(a, nbv, lk, s, acc);
  hop_pair<St, R, LT, 3, SF, PASS == PASS_A && MOB>(a, nbv, lk, s, acc);

  double nrm2 = 0.0;
  if (PASS == PASS_A) {
    apply_minv<R, false>(acc, s, a);
    if (MOB) {
      apply_lin<R, false>(acc, (R)a.b, (R)a.c, s, a.Ls, m);
    } else {
      const R bb = (R)(a.b * a.b);
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] *= bb;
    }
  } else if (PASS == PASS_C) {
    if (MOB) {
      apply_lin<R, true>(acc, (R)a.b, (R)a.c, s, a.Ls, m);
    } else {
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] *= (R)a.b;
    }
    apply_minv<R, true>(acc, s, a);
  } else {
    // B, D: out = M_oo^(dag) in2 - K^(dag) acc / 4   (B has no K on this side)
    if (PASS == PASS_D) {
      if (MOB) {
        apply_lin<R, true>(acc, (R)a.b, (R)a.c, s, a.Ls, m);
      } else {
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] *= (R)a.b;
      }
    }
    R self[24];
    load_spinor<St, R>(a.in2, site5, a.n5, self);
    apply_lin<R, DAG>(self, (R)a.alpha, (R)a.beta, s, a.Ls, m);
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = self[i] - R(0.25) * acc[i];
    if (PASS == PASS_D) {
      const R sD = (R)a.sD;
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] *= sD;
      if (a.extra) {
        R ex[24];
        load_spinor<St, R>(a.extra, site5, a.n5, ex);
        const R lam = (R)a.lam;
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] += lam * ex[i];
      }
    }
  }
  if (active) store_spinor<St, R>(a.out, site5, a.n5, acc);
  if (a.do_red) {
    if (active) {
      R t = 0;
#pragma unroll
      for (int i = 0; i < 24; ++i) t += acc[i] * acc[i];
      nrm2 = (double)t;
    }
    double v[1] = {nrm2};
    grid_reduce<1>(v, a.red);
  }
}

// ------------------------------------------------------------------------------
// tables and gauge field
// ------------------------------------------------------------------------------
struct Geom {
  int L[4];
  int parity;
  size_t n4;
};

__device__ __forceinline__ void cb_coords(const Geom& g, size_t i, int* x) {
  const int hx = g.L[0] / 2;
  size_t rest = i / hx;
  x[1] = (int)(rest % g.L[1]);
  rest /= g.L[1];
  x[2] = (int)(rest % g.L[2]);
  x[3] = (int)(rest / g.L[2]);
  const int delta = (g.parity + x[1] + x[2] + x[3]) & 1;
  x[0] = 2 * (int)(i % hx) + delta;
}

__device__ __forceinline__ size_t lex_of(const Geom& g, const int* x) {
  return (size_t)x[0] + (size_t)g.L[0] * (x[1] + (size_t)g.L[1] * (x[2] + (size_t)g.L[2] * x[3]));
}

__global__ void nbr_kernel(Geom g, int* nbr) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n4) return;
  int x[4];
  cb_coords(g, i, x);
  for (int dir = 0; dir < 8; ++dir) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    const int mu = dir & 3;
    y[mu] = (y[mu] + (dir < 4 ? 1 : g.L[mu] - 1)) % g.L[mu];
    nbr[i * 8 + dir] = (int)(lex_of(g, y) >> 1);
  }
}

// links[p][i][dir][3][3]: dir < 4: U_mu(x); dir >= 4: U_mu(x - mu)^dag; the
// antiperiodic time boundary is folded in as a sign.
__global__ void link_kernel(Geom g, int apbc, const double2* __restrict__ U, double2* l64,
                            float2* l32, __half2* l16, __nv_bfloat162* lb16) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n4) return;
  int x[4];
  cb_coords(g, i, x);
  for (int dir = 0; dir < 8; ++dir) {
    const int mu = dir & 3;
    int y[4] = {x[0], x[1], x[2], x[3]};
    double sign = 1.0;
    if (dir >= 4) {
      y[mu] = (y[mu] + g.L[mu] - 1) % g.L[mu];
      if (apbc && mu == 3 && x[3] == 0) sign = -1.0;
    } else {
      if (apbc && mu == 3 && x[3] == g.L[3] - 1) sign = -1.0;
    }
    const double2* src = U + (lex_of(g, y) * 4 + mu) * 9;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double2 v = dir < 4 ? src[r * 3 + c] : src[c * 3 + r];
        if (dir >= 4) v.y = -v.y;
        v.x *= sign;
        v.y *= sign;
        const size_t o = (i * 8 + dir) * 9 + r * 3 + c;
        l64[o] = v;
        l32[o] = make_float2((float)v.x, (float)v.y);
        l16[o] = __floats2half2_rn((float)v.x, (float)v.y);
        lb16[o] = __floats2bfloat162_rn((float)v.x, (float)v.y);
      }
  }
}

static Geom geom(const Ctx& c, int parity) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = c.dims[i];
  g.parity = parity;
  g.n4 = c.n4;
  return g;
}

void dwf_setup_tables(Ctx& c) {
  for (int p = 0; p < 2; ++p) {
    c.nbr[p].ensure(c.n4 * 8 * sizeof(int));
    nbr_kernel<<<(unsigned)((c.n4 + 255) / 256), 256, 0, c.stream>>>(geom(c, p), c.nbr[p].as<int>());
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
  }
}

void dwf_upload_gauge(Ctx& c, const void* U, bool on_device) {
  const size_t canon = c.V * 4 * 9 * sizeof(double2);
  const double2* src = reinterpret_cast<const double2*>(U);
  DevMem tmp;
  if (!on_device) {
    tmp.ensure(canon);
    HDCG_CUDA(cudaMemcpyAsync(tmp.p, U, canon, cudaMemcpyHostToDevice, c.stream));
    src = tmp.as<double2>();
  }
  const size_t nl = c.n4 * 8 * 9;
  for (int p = 0; p < 2; ++p) {
    c.links[HDCG_F64][p].ensure(nl * sizeof(double2));
    c.links[HDCG_F32][p].ensure(nl * sizeof(float2));
    c.links[HDCG_F16][p].ensure(nl * sizeof(__half2));
    c.links[HDCG_BF16][p].ensure(nl * sizeof(__nv_bfloat162));
    link_kernel<<<(unsigned)((c.n4 + 255) / 256), 256, 0, c.stream>>>(
        geom(c, p), c.apbc, src, c.links[HDCG_F64][p].as<double2>(), c.links[HDCG_F32][p].as<float2>(),
        c.links[HDCG_F16][p].as<__half2>(), c.links[HDCG_BF16][p].as<__nv_bfloat162>());
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
  }
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  c.have_gauge = true;
}

void dwf_set_coeffs(Ctx& c, double M5, double b, double cc, double mass) {
  DwfCoeffs& k = c.co;
  k.M5 = M5;
  k.b = b;
  k.c = cc;
  k.mass = mass;
  k.alpha = b * (4.0 - M5) + 1.0;
  k.beta = cc * (4.0 - M5) - 1.0;
  HDCG_REQUIRE(std::fabs(k.alpha) > 1e-300, HDCG_ERR_ARG, "b (4 - M5) + 1 must be nonzero");
  k.minv_r = -k.beta / k.alpha;
  const double denom = k.alpha * (1.0 + mass * std::pow(k.minv_r, c.Ls));
  HDCG_REQUIRE(std::fabs(denom) > 1e-300 && std::isfinite(denom), HDCG_ERR_ARG, "M_ee is singular");
  k.minv_norm = 1.0 / denom;
  double r = k.minv_r;
  for (int j = 0; j < 6; ++j) {
    k.rpow[j] = r;
    r = r * r;
  }
  c.have_dwf = true;
}

// ------------------------------------------------------------------------------
// launches
// ------------------------------------------------------------------------------
template <typename St>
static void launch_typed(int pass, bool mob, const HopArgs& a, unsigned grid, cudaStream_t st) {
#define HDCG_HOP_CASE(P)                                                         \
  if (pass == P) {                                                               \
    if (mob) hop_kernel<St, P, true><<<grid, 256, 0, st>>>(a);                   \
    else hop_kernel<St, P, false><<<grid, 256, 0, st>>>(a);                      \
    return;                                                                      \
  }
  HDCG_HOP_CASE(PASS_A)
  HDCG_HOP_CASE(PASS_B)
  HDCG_HOP_CASE(PASS_C)
  HDCG_HOP_CASE(PASS_D)
#undef HDCG_HOP_CASE
}

static double hop_bytes(const Ctx& c, int pass, int prec, bool extra) {
  const double fb = (double)bytes_per_real(prec);
  const double lb = (double)bytes_per_real(prec);  // link reals stored in the field precision
  double reals_field = 48.0 + ((pass == PASS_B || pass == PASS_D) ? 24.0 : 0.0) + (extra ? 24.0 : 0.0);
  return (double)c.n5 * (reals_field * fb + 8.0 * 18.0 * lb / c.Ls);
}

void launch_hop(Ctx& c, int pass, int prec, const uint4* in, const uint4* in2, uint4* out,
                const HopEpi& epi, double* red_result, int accumulate) {
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  const int out_par = (pass == PASS_A || pass == PASS_C) ? 0 : 1;
  HopArgs a;
  a.in = in;
  a.in2 = in2;
  a.extra = epi.extra;
  a.out = out;
  a.links = c.links[link_slot(prec)][out_par].p;
  a.nbr = c.nbr[out_par].as<int>();
  a.n5 = c.n5;
  a.Ls = c.Ls;
  a.lslog2 = c.lslog2;
  a.b = c.co.b;
  a.c = c.co.c;
  a.alpha = c.co.alpha;
  a.beta = c.co.beta;
  a.mass = c.co.mass;
  a.minv_norm = c.co.minv_norm;
  for (int j = 0; j < 6; ++j) a.rpow[j] = c.co.rpow[j];
  a.sD = epi.sD;
  a.lam = epi.lam;
  const unsigned grid = (unsigned)((c.n5 + 255) / 256);
  a.do_red = red_result != nullptr;
  if (a.do_red) {
    c.red_partials.ensure((size_t)grid * 4 * sizeof(double));
    a.red.partials = c.red_partials.as<double>();
    a.red.ticket = c.red_ticket.as<unsigned>();
    a.red.result = red_result;
    a.red.accumulate = accumulate;
  }
  const bool mob = c.co.c != 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c.prof.on) {
    HDCG_CUDA(cudaEventCreate(&ev0));
    HDCG_CUDA(cudaEventCreate(&ev1));
    HDCG_CUDA(cudaEventRecord(ev0, c.stream));
  }
  switch (prec) {
    case HDCG_F64: launch_typed<f64_t>(pass, mob, a, grid, c.stream); break;
    case HDCG_F32: launch_typed<f32_t>(pass, mob, a, grid, c.stream); break;
    case HDCG_F16: launch_typed<f16_t>(pass, mob, a, grid, c.stream); break;
    case HDCG_BF16: launch_typed<bf16_t>(pass, mob, a, grid, c.stream); break;
    case HDCG_BF16T: launch_typed<bf16t_t>(pass, mob, a, grid, c.stream); break;
    default: throw Error{HDCG_ERR_ARG, "unknown precision code"};
  }
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  if (c.prof.on) {
    HDCG_CUDA(cudaEventRecord(ev1, c.stream));
    c.prof.pending.push_back(ev0);
    c.prof.pending.push_back(ev1);
    c.prof.pending_prec.push_back(prec);
    c.prof.bytes[prec] += hop_bytes(c, pass, prec, epi.extra != nullptr);
  }
}

void apply_mpc(Ctx& c, int prec, const uint4* in, uint4* out, int dagger, double* mpc_norm2) {
  uint4* t = c.scratch(prec, 0);
  if (!dagger) {
    launch_hop(c, PASS_A, prec, in, nullptr, t, HopEpi{}, nullptr, 0);
    launch_hop(c, PASS_B, prec, t, in, out, HopEpi{}, mpc_norm2, 0);
  } else {
    launch_hop(c, PASS_C, prec, in, nullptr, t, HopEpi{}, nullptr, 0);
    launch_hop(c, PASS_D, prec, t, in, out, HopEpi{}, nullptr, 0);
  }
}

void apply_mdagm(Ctx& c, int prec, const uint4* in, uint4* out, double* mpc_norm2, double sD,
                 double lam, const uint4* extra) {
  uint4* t = c.scratch(prec, 0);
  uint4* chi = c.scratch(prec, 1);
  launch_hop(c, PASS_A, prec, in, nullptr, t, HopEpi{}, nullptr, 0);
  launch_hop(c, PASS_B, prec, t, in, chi, HopEpi{}, mpc_norm2, 0);
  launch_hop(c, PASS_C, prec, chi, nullptr, t, HopEpi{}, nullptr, 0);
  HopEpi e;
  e.sD = sD;
  e.lam = lam;
  e.extra = extra;
  launch_hop(c, PASS_D, prec, t, chi, out, e, nullptr, 0);
}

}  // namespace hdcg
