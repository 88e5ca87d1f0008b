// Device code of the fine-operator hop passes (see dwf.cu for the operator).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "context.h"
#include "dfloat.cuh"

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
  // the same coefficients rounded to float on the host: the FP32/16-bit passes
  // read these, so no thread converts from double (GB300's FP64 pipe is narrow)
  float fb, fc, falpha, fbeta, fmass, fminv_norm, frpow[6], fsD, flam;
  Reduction red;
  int do_red;
  // fused CG step in pass D (cg_r != null): w = out is not stored; instead
  // alpha = *al_num / (*al_den0 + al_lam * *al_den1), r -= alpha w, x += alpha p,
  // and the reduction receives |r|^2
  uint4* cg_x;
  uint4* cg_r;
  const uint4* cg_p;
  const double* al_num;
  const double* al_den0;
  const double* al_den1;
  double al_lam;
  // several right-hand sides (grid y): fields fstride granules apart, the
  // fused-CG scalars of right-hand side r at al_*[r]; al_mask[r] == 0 freezes r
  size_t fstride;
  const int* al_mask;
};

// coefficient in the arithmetic type R: the host-rounded float for FP32
// arithmetic, the double otherwise (FP64 and double-float passes)
template <typename R> __device__ __forceinline__ R sc(double d, float) { return R(d); }
template <> __device__ __forceinline__ float sc<float>(double, float f) { return f; }

// ------------------------------------------------------------------------------
// link loads: 9 complex of one link into 18 reals.  Links are stored padded to
// whole 16-byte granules (LINK_GRAN[prec] granules per link) so that one link
// is read with 16-byte loads: FP64 9, FP32 5, 16-bit 3 granules.
// ------------------------------------------------------------------------------
template <typename LT> struct LinkGran;
template <> struct LinkGran<double2> { static constexpr int g = 9; };
template <> struct LinkGran<float4> { static constexpr int g = 9; };   // double-float (re hi, re lo, im hi, im lo)
template <> struct LinkGran<float2> { static constexpr int g = 5; };
template <> struct LinkGran<__half2> { static constexpr int g = 3; };
template <> struct LinkGran<__nv_bfloat162> { static constexpr int g = 3; };

__device__ __forceinline__ void load_link(const double2*, const uint4* __restrict__ p, double* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint4 g = __ldg(p + i);
    u[2 * i] = __hiloint2double(g.y, g.x);
    u[2 * i + 1] = __hiloint2double(g.w, g.z);
  }
}
__device__ __forceinline__ void load_link(const float4*, const uint4* __restrict__ p, dfl* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint4 g = __ldg(p + i);
    u[2 * i] = dfl(__uint_as_float(g.x), __uint_as_float(g.y));
    u[2 * i + 1] = dfl(__uint_as_float(g.z), __uint_as_float(g.w));
  }
}
__device__ __forceinline__ void load_link(const double2*, const uint4* __restrict__ p, dfl* u) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint4 g = __ldg(p + i);
    u[2 * i] = dfl(__hiloint2double(g.y, g.x));
    u[2 * i + 1] = dfl(__hiloint2double(g.w, g.z));
  }
}
__device__ __forceinline__ void load_link(const float2*, const uint4* __restrict__ p, float* u) {
  // 8-byte loads keep the register footprint of the FP32 kernels low
  const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float2 v = __ldg(q + i);
    u[2 * i] = v.x;
    u[2 * i + 1] = v.y;
  }
}
template <typename H2>
__device__ __forceinline__ void load_link16(const uint4* __restrict__ p, float* u, bool bf) {
  unsigned t[12];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const uint4 g = __ldg(p + i);
    t[4 * i] = g.x;
    t[4 * i + 1] = g.y;
    t[4 * i + 2] = g.z;
    t[4 * i + 3] = g.w;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float2 v = bf ? b2f(t[i]) : h2f(t[i]);
    u[2 * i] = v.x;
    u[2 * i + 1] = v.y;
  }
}
__device__ __forceinline__ void load_link(const __half2*, const uint4* __restrict__ p, float* u) {
  load_link16<__half2>(p, u, false);
}
__device__ __forceinline__ void load_link(const __nv_bfloat162*, const uint4* __restrict__ p, float* u) {
  load_link16<__nv_bfloat162>(p, u, true);
}

// ------------------------------------------------------------------------------
// s-direction operators on one lane's 24 reals; spins 0,1 are chirality +
// (gamma5 = +1), spins 2,3 chirality -.  P_s acts on chirality + as the down
// shift (psi_{s-1}) and on chirality - as the up shift (psi_{s+1}); P_s^dag
// swaps them.  Wrapped values pick up -m.
// ------------------------------------------------------------------------------
// Each element shuffles only itself, so the shift-and-combine steps below
// update v in place (every lane reads its source lane's old value in the same
// warp-wide shuffle) with the wall factor folded into one coefficient per
// chirality: one shuffle and one multiply-add per real.

// v <- a v + b P v
template <typename R, bool DAG>
__device__ __forceinline__ void apply_lin(R* v, R a, R b, int s, int Ls, R m) {
  const int up_src = (s + 1) & (Ls - 1), dn_src = (s - 1) & (Ls - 1);
  const R up_f = (s + 1 >= Ls) ? -m : R(1), dn_f = (s < 1) ? -m : R(1);
  const int sp = DAG ? up_src : dn_src, sm = DAG ? dn_src : up_src;
  const R bp = b * (DAG ? up_f : dn_f), bm = b * (DAG ? dn_f : up_f);
#pragma unroll
  for (int i = 0; i < 12; ++i) v[i] = a * v[i] + bp * shfl_any(v[i], sp, Ls);
#pragma unroll
  for (int i = 12; i < 24; ++i) v[i] = a * v[i] + bm * shfl_any(v[i], sm, Ls);
}

// v <- M_ee^-1 v (DAG: M_ee^-dag) by doubling: A_{j+1} = A_j + r^{2^j} P^{2^j} A_j
template <typename R, bool DAG>
__device__ __forceinline__ void apply_minv(R* v, int s, const HopArgs& a) {
  const R m = sc<R>(a.mass, a.fmass);
  const int Ls = a.Ls;
  for (int j = 0; j < a.lslog2; ++j) {
    const int d = 1 << j;
    const int up_src = (s + d) & (Ls - 1), dn_src = (s - d) & (Ls - 1);
    const R up_f = (s + d >= Ls) ? -m : R(1), dn_f = (s < d) ? -m : R(1);
    const int sp = DAG ? up_src : dn_src, sm = DAG ? dn_src : up_src;
    const R rp = sc<R>(a.rpow[j], a.frpow[j]);
    const R cp = rp * (DAG ? up_f : dn_f), cm = rp * (DAG ? dn_f : up_f);
#pragma unroll
    for (int i = 0; i < 12; ++i) v[i] += cp * shfl_any(v[i], sp, Ls);
#pragma unroll
    for (int i = 12; i < 24; ++i) v[i] += cm * shfl_any(v[i], sm, Ls);
  }
  const R nrm = sc<R>(a.minv_norm, a.fminv_norm);
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
template <> struct LinkOf<df_t> { using T = float4; };
template <> struct LinkOf<f32_t> { using T = float2; };
template <> struct LinkOf<f16_t> { using T = __half2; };
template <> struct LinkOf<bf16_t> { using T = __nv_bfloat162; };
template <> struct LinkOf<bf16t_t> { using T = __nv_bfloat162; };

// both hops along direction MU: forward (x + mu, projector 1 - SF g) and
// backward (x - mu, projector 1 + SF g); the two neighbour spinors and links are
// loaded before either is used so that their loads overlap.
template <typename St, typename R, typename LT, int MU, int SF, bool KIN>
__device__ __forceinline__ void hop_pair(const HopArgs& a, const uint4* in, const int* nbv, const uint4* lk, int s,
                                         R* acc) {
  constexpr int LG = LinkGran<LT>::g;
  if constexpr (std::is_same<R, dfl>::value) {
    // double-float: compute-bound, so one neighbour at a time keeps registers low
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      R ps[24];
      load_spinor<St, R>(in, (size_t)nbv[MU + 4 * side] * a.Ls + s, a.n5, ps);
      if (KIN) apply_lin<R, false>(ps, sc<R>(a.b, a.fb), sc<R>(a.c, a.fc), s, a.Ls, sc<R>(a.mass, a.fmass));
      R h[12], uh[12], U[18];
      load_link((const LT*)nullptr, lk + (MU + 4 * side) * LG, U);
      if (side == 0) {
        project<MU, SF>(ps, h);
        su3_mul<R>(U, h, uh);
        reconstruct_add<MU, SF>(uh, acc);
      } else {
        project<MU, -SF>(ps, h);
        su3_mul<R>(U, h, uh);
        reconstruct_add<MU, -SF>(uh, acc);
      }
    }
  } else {
    R pf[24], pb[24];
    load_spinor<St, R>(in, (size_t)nbv[MU] * a.Ls + s, a.n5, pf);
    load_spinor<St, R>(in, (size_t)nbv[MU + 4] * a.Ls + s, a.n5, pb);
    if (KIN) {
      const R m = sc<R>(a.mass, a.fmass), kb = sc<R>(a.b, a.fb), kc = sc<R>(a.c, a.fc);
      apply_lin<R, false>(pf, kb, kc, s, a.Ls, m);
      apply_lin<R, false>(pb, kb, kc, s, a.Ls, m);
    }
    R h[12], uh[12], U[18];
    project<MU, SF>(pf, h);
    load_link((const LT*)nullptr, lk + MU * LG, U);
    su3_mul<R>(U, h, uh);
    reconstruct_add<MU, SF>(uh, acc);
    project<MU, -SF>(pb, h);
    load_link((const LT*)nullptr, lk + (MU + 4) * LG, U);
    su3_mul<R>(U, h, uh);
    reconstruct_add<MU, -SF>(uh, acc);
  }
}

// hop along MU from raw (already loaded) 16-bit granules of the neighbours
template <typename St, typename R, typename LT, int MU, int SF, bool KIN>
__device__ __forceinline__ void hop_raw(const HopArgs& a, const uint4 (&raw)[8][3], const uint4* lk, int s, R* acc) {
  constexpr int LG = LinkGran<LT>::g;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    R ps[24];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float t[8];
      unpack(St{}, raw[MU + 4 * side][c], t);
#pragma unroll
      for (int i = 0; i < 8; ++i) ps[c * 8 + i] = (R)t[i];
    }
    if (KIN) apply_lin<R, false>(ps, sc<R>(a.b, a.fb), sc<R>(a.c, a.fc), s, a.Ls, sc<R>(a.mass, a.fmass));
    R h[12], uh[12], U[18];
    load_link((const LT*)nullptr, lk + (MU + 4 * side) * LG, U);
    if (side == 0) {
      project<MU, SF>(ps, h);
      su3_mul<R>(U, h, uh);
      reconstruct_add<MU, SF>(uh, acc);
    } else {
      project<MU, -SF>(ps, h);
      su3_mul<R>(U, h, uh);
      reconstruct_add<MU, -SF>(uh, acc);
    }
  }
}

// |acc|^2 of the pass into the FP64 grid reduction.  FP32 arithmetic: each
// warp sums its lanes' float partials by double-float TwoSum steps on the FP32
// pipes (about 48 bits) and only the per-warp totals are added in FP64; the
// FP64 and double-float passes reduce in FP64 throughout.
template <typename R>
__device__ __forceinline__ void hop_norm2(const R* acc, bool active, const Reduction& red) {
  if constexpr (std::is_same<R, float>::value) {
    float t = 0.f;
    if (active) {
#pragma unroll
      for (int i = 0; i < 24; ++i) t = fmaf(acc[i], acc[i], t);
    }
    float hi = t, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(FULL_MASK, hi, o), ol = __shfl_xor_sync(FULL_MASK, lo, o);
      float sh, eh;
      two_sum(hi, oh, sh, eh);
      eh = __fadd_rn(eh, __fadd_rn(lo, ol));
      fast_two_sum(sh, eh, hi, lo);
    }
    double v[1] = {(double)hi + (double)lo};
    grid_reduce<1, true>(v, red);
  } else {
    double nrm2 = 0.0;
    if (active) {
      R t = 0;
#pragma unroll
      for (int i = 0; i < 24; ++i) t += acc[i] * acc[i];
      nrm2 = (double)t;
    }
    double v[1] = {nrm2};
    grid_reduce<1>(v, red);
  }
}

// ------------------------------------------------------------------------------
// one hop pass
// ------------------------------------------------------------------------------
// Arithmetic type of the hop passes: FP32 for 16/32-bit storage; double-float
// (about 48 bits, on the FP32 pipes) for FP64 storage.
// arithmetic type of the hop: float for FP32/16-bit storage; for FP64 storage
// either native double or (DF) a double-float pair on the FP32 pipes
template <typename St, bool DF> struct HopCompute { using type = float; };
template <> struct HopCompute<f64_t, false> { using type = double; };
template <> struct HopCompute<f64_t, true> { using type = dfl; };
template <bool DF> struct HopCompute<df_t, DF> { using type = dfl; };

// MINB: minimum resident CTAs per SM requested from the compiler (register
// budget); the variants are chosen at run time by the hop autotuner.
// PF (16-bit storage only): the raw 16-byte granules of all eight neighbour
// spinors are loaded before any is used (24 loads in flight per thread).
// DF (FP64 storage only): double-float arithmetic instead of FP64 units.
template <typename St, int PASS, bool MOB, int MINB, bool PF = false, bool DF = false>
__global__ void __launch_bounds__(256, MINB) hop_kernel(const HopArgs a) {
  using R = typename HopCompute<St, DF>::type;
  using LT = typename LinkOf<St>::T;
  constexpr bool DAG = (PASS == PASS_C || PASS == PASS_D);
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gtid < a.n5;
  const size_t roff = (size_t)blockIdx.y * a.fstride;  // right-hand side offset (granules)
  const int rhs = blockIdx.y;
  const int s = threadIdx.x & (a.Ls - 1);
  const size_t x4 = active ? (gtid >> a.lslog2) : 0;
  const size_t site5 = x4 * a.Ls + s;
  const R m = sc<R>(a.mass, a.fmass);
  const R kb = sc<R>(a.b, a.fb), kc = sc<R>(a.c, a.fc);

  R acc[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = 0;

  const uint4* in = a.in + roff;
  // all eight neighbour indices at once (32 bytes, shared by the Ls lanes of a site)
  const int4 nb0 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2);
  const int4 nb1 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2 + 1);
  const int nbv[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};
  const uint4* lk = reinterpret_cast<const uint4*>(a.links) + x4 * 8 * LinkGran<LT>::g;
  // Dh: forward (1 - g), backward (1 + g); Dh^dag flips both.
  constexpr int SF = DAG ? -1 : 1;
  if constexpr (PF && Store<St>::chunks == 3) {
    uint4 raw[8][3];
#pragma unroll
    for (int d = 0; d < 8; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c) raw[d][c] = __ldg(in + c * a.n5 + (size_t)nbv[d] * a.Ls + s);
    hop_raw<St, R, LT, 0, SF, PASS == PASS_A && MOB>(a, raw, lk, s, acc);
    hop_raw<St, R, LT, 1, SF, PASS == PASS_A && MOB>(a, raw, lk, s, acc);
    hop_raw<St, R, LT, 2, SF, PASS == PASS_A && MOB>(a, raw, lk, s, acc);
    hop_raw<St, R, LT, 3, SF, PASS == PASS_A && MOB>(a, raw, lk, s, acc);
  } else {
    hop_pair<St, R, LT, 0, SF, PASS == PASS_A && MOB>(a, in, nbv, lk, s, acc);
    hop_pair<St, R, LT, 1, SF, PASS == PASS_A && MOB>(a, in, nbv, lk, s, acc);
    hop_pair<St, R, LT, 2, SF, PASS == PASS_A && MOB>(a, in, nbv, lk, s, acc);
    hop_pair<St, R, LT, 3, SF, PASS == PASS_A && MOB>(a, in, nbv, lk, s, acc);
  }

  if (PASS == PASS_A) {
    apply_minv<R, false>(acc, s, a);
    if (MOB) {
      apply_lin<R, false>(acc, kb, kc, s, a.Ls, m);
    } else {
      const R bb = kb * kb;
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] *= bb;
    }
  } else if (PASS == PASS_C) {
    if (MOB) {
      apply_lin<R, true>(acc, kb, kc, s, a.Ls, m);
    } else {
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] *= kb;
    }
    apply_minv<R, true>(acc, s, a);
  } else {
    // B, D: out = M_oo^(dag) in2 - K^(dag) acc / 4   (B has no K on this side)
    if (PASS == PASS_D) {
      if (MOB) {
        apply_lin<R, true>(acc, kb, kc, s, a.Ls, m);
      } else {
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] *= kb;
      }
    }
    R self[24];
    load_spinor<St, R>(a.in2 + roff, site5, a.n5, self);
    apply_lin<R, DAG>(self, sc<R>(a.alpha, a.falpha), sc<R>(a.beta, a.fbeta), s, a.Ls, m);
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = self[i] - R(0.25) * acc[i];
    if (PASS == PASS_D) {
      const R sD = sc<R>(a.sD, a.fsD);
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] *= sD;
      if (a.extra) {
        R ex[24];
        load_spinor<St, R>(a.extra + roff, site5, a.n5, ex);
        const R lam = sc<R>(a.lam, a.flam);
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] += lam * ex[i];
      }
    }
  }
  if (PASS == PASS_D && a.cg_r) {
    // alpha of the fused CG step: one FP64 division per CTA, shared
    __shared__ double s_alpha;
    __shared__ float s_alphaf;
    if (threadIdx.x == 0) {
      double den = a.al_den0[rhs];
      if (a.al_den1) den += a.al_lam * a.al_den1[rhs];
      const bool live = a.al_mask == nullptr || a.al_mask[rhs] != 0;
      s_alpha = (den != 0.0 && live) ? a.al_num[rhs] / den : 0.0;
      s_alphaf = (float)s_alpha;
    }
    __syncthreads();
    const R alpha = sc<R>(s_alpha, s_alphaf);
    if (active) {
      R rv[24], xv[24], pv[24];
      load_spinor<St, R>(a.cg_r + roff, site5, a.n5, rv);
      load_spinor<St, R>(a.cg_x + roff, site5, a.n5, xv);
      load_spinor<St, R>(a.cg_p + roff, site5, a.n5, pv);
#pragma unroll
      for (int i = 0; i < 24; ++i) {
        rv[i] -= alpha * acc[i];
        xv[i] += alpha * pv[i];
        acc[i] = rv[i];
      }
      store_spinor<St, R>(a.cg_r + roff, site5, a.n5, rv);
      store_spinor<St, R>(a.cg_x + roff, site5, a.n5, xv);
    }
  } else if (active) {
    store_spinor<St, R>(a.out + roff, site5, a.n5, acc);
  }
  if (a.do_red) hop_norm2<R>(acc, active, a.red);
}


}  // namespace hdcg

#include "hop_packed.cuh"

namespace hdcg {

// MINB = 1, 2, 3; 4th (MINB 1): prefetch of all neighbours for 16-bit storage,
// double-float arithmetic for FP64 storage; 5th and 6th (FP32 and 16-bit
// storage only): packed FP32 arithmetic (hop_packed.cuh) with MINB 2 and 1
constexpr int HOP_VARIANTS = 6;
template <typename St> constexpr int hop_variants() { return Store<St>::chunks == 12 ? 4 : 6; }

// launch variant v of one pass for storage St
template <typename St>
void launch_hop_variant(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st) {
  if constexpr (Store<St>::chunks != 12) {
    if (v >= 4) {
      const bool stage = a.Ls >= 8;
#define HDCG_HOP_PK(P, M)                                                                       \
      if (pass == P) {                                                                         \
        if (stage) {                                                                           \
          if (mob) pk::hop_packed_kernel<St, P, true, M, true><<<grid, 256, 0, st>>>(a);       \
          else pk::hop_packed_kernel<St, P, false, M, true><<<grid, 256, 0, st>>>(a);          \
        } else {                                                                               \
          if (mob) pk::hop_packed_kernel<St, P, true, M, false><<<grid, 256, 0, st>>>(a);      \
          else pk::hop_packed_kernel<St, P, false, M, false><<<grid, 256, 0, st>>>(a);         \
        }                                                                                      \
        return;                                                                                \
      }
      if (v == 4) {
        HDCG_HOP_PK(PASS_A, 2) HDCG_HOP_PK(PASS_B, 2) HDCG_HOP_PK(PASS_C, 2) HDCG_HOP_PK(PASS_D, 2)
      } else {
        HDCG_HOP_PK(PASS_A, 1) HDCG_HOP_PK(PASS_B, 1) HDCG_HOP_PK(PASS_C, 1) HDCG_HOP_PK(PASS_D, 1)
      }
#undef HDCG_HOP_PK
      return;
    }
  }
#define HDCG_HOP_CASE(P, M)                                                      \
  if (pass == P && v == M - 1) {                                                 \
    if (mob) hop_kernel<St, P, true, M><<<grid, 256, 0, st>>>(a);               \
    else hop_kernel<St, P, false, M><<<grid, 256, 0, st>>>(a);                  \
    return;                                                                      \
  }
  HDCG_HOP_CASE(PASS_A, 1) HDCG_HOP_CASE(PASS_A, 2) HDCG_HOP_CASE(PASS_A, 3)
  HDCG_HOP_CASE(PASS_B, 1) HDCG_HOP_CASE(PASS_B, 2) HDCG_HOP_CASE(PASS_B, 3)
  HDCG_HOP_CASE(PASS_C, 1) HDCG_HOP_CASE(PASS_C, 2) HDCG_HOP_CASE(PASS_C, 3)
  HDCG_HOP_CASE(PASS_D, 1) HDCG_HOP_CASE(PASS_D, 2) HDCG_HOP_CASE(PASS_D, 3)
#undef HDCG_HOP_CASE
  if (v == 3) {
    constexpr bool PF = Store<St>::chunks == 3;
    constexpr bool DF = Store<St>::chunks == 12;
#define HDCG_HOP_PF(P)                                                           \
    if (pass == P) {                                                             \
      if (mob) hop_kernel<St, P, true, 1, PF, DF><<<grid, 256, 0, st>>>(a);     \
      else hop_kernel<St, P, false, 1, PF, DF><<<grid, 256, 0, st>>>(a);        \
      return;                                                                    \
    }
    HDCG_HOP_PF(PASS_A) HDCG_HOP_PF(PASS_B) HDCG_HOP_PF(PASS_C) HDCG_HOP_PF(PASS_D)
#undef HDCG_HOP_PF
  }
}

// explicit instantiations live in dwf_<prec>.cu
void launch_hop_f64(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st);
void launch_hop_f32(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st);
void launch_hop_f16(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st);
void launch_hop_bf16(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st);
void launch_hop_bf16t(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st);
void launch_hop_df(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st);

}  // namespace hdcg
