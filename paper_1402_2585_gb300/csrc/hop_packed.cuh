// Fine-operator hop passes with packed FP32 arithmetic (FP32 and 16-bit storage).
//
// Same operator and pass structure as hop_kernel (dwf_kernels.cuh); only the
// arithmetic is arranged differently.  On sm_100-class GPUs the FMA pipe
// executes add / mul / fma on a pair of floats per instruction (f32x2), so a
// complex number kept as one (re, im) register pair costs one instruction per
// complex add, and a complex multiply-accumulate costs two:
//   acc += u h  =  (u_re, u_re) (h_re, h_im) + (-u_im, u_im) (h_im, h_re) + acc.
// The gauge links of a CTA's 4D sites are read once, converted to FP32 and
// expanded to these (u_re, u_re, -u_im, u_im) quadruples in shared memory; the
// Ls lanes of a 4D site then read them as one 16-byte shared load per entry.
// Multiplications by +-i (spin projection and reconstruction along x and z)
// swap the two halves of a pair.
#pragma once

namespace hdcg {
namespace pk {

typedef unsigned long long c2;   // (re, im): low word re, high word im

__device__ __forceinline__ c2 make(float re, float im) {
  c2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(re), "f"(im));
  return r;
}
__device__ __forceinline__ void split(c2 a, float& re, float& im) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(re), "=f"(im) : "l"(a));
}
__device__ __forceinline__ c2 add(c2 a, c2 b) {
  c2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ c2 sub(c2 a, c2 b) {
  c2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ c2 mul(c2 a, c2 b) {
  c2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// a b + c, elementwise
__device__ __forceinline__ c2 fma(c2 a, c2 b, c2 c) {
  c2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ c2 bc(float x) { return make(x, x); }
// (im, re)
__device__ __forceinline__ c2 swp(c2 a) {
  float r, i;
  split(a, r, i);
  return make(i, r);
}
__device__ __forceinline__ c2 shfl(c2 a, int src, int width) {
  float r, i;
  split(a, r, i);
  return make(__shfl_sync(FULL_MASK, r, src, width), __shfl_sync(FULL_MASK, i, src, width));
}

// 12 complex (spin-major: index spin * 3 + colour) of one site in the chunked layout
__device__ __forceinline__ c2 h2c(unsigned v) {
  const float2 f = h2f(v);
  return make(f.x, f.y);
}
__device__ __forceinline__ c2 b2c(unsigned v) {
  const float2 f = b2f(v);
  return make(f.x, f.y);
}
__device__ __forceinline__ void unpack_c(f32_t, const uint4& g, c2* v) {
  v[0] = make(__uint_as_float(g.x), __uint_as_float(g.y));
  v[1] = make(__uint_as_float(g.z), __uint_as_float(g.w));
}
__device__ __forceinline__ void unpack_c(f16_t, const uint4& g, c2* v) {
  v[0] = h2c(g.x);
  v[1] = h2c(g.y);
  v[2] = h2c(g.z);
  v[3] = h2c(g.w);
}
__device__ __forceinline__ void unpack_c(bf16_t, const uint4& g, c2* v) {
  v[0] = b2c(g.x);
  v[1] = b2c(g.y);
  v[2] = b2c(g.z);
  v[3] = b2c(g.w);
}
__device__ __forceinline__ void unpack_c(bf16t_t, const uint4& g, c2* v) { unpack_c(bf16_t{}, g, v); }

template <typename St>
__device__ __forceinline__ void load_raw(const uint4* __restrict__ f, size_t site5, size_t n5,
                                         uint4 (&g)[Store<St>::chunks]) {
#pragma unroll
  for (int c = 0; c < Store<St>::chunks; ++c) g[c] = __ldg(f + c * n5 + site5);
}
template <typename St>
__device__ __forceinline__ void unpack_site(const uint4 (&g)[Store<St>::chunks], c2* v) {
  constexpr int PC = Store<St>::per_chunk / 2;   // complex per granule
#pragma unroll
  for (int c = 0; c < Store<St>::chunks; ++c) unpack_c(St{}, g[c], v + c * PC);
}
template <typename St>
__device__ __forceinline__ void load_c(const uint4* __restrict__ f, size_t site5, size_t n5, c2* v) {
  uint4 g[Store<St>::chunks];
  load_raw<St>(f, site5, n5, g);
  unpack_site<St>(g, v);
}

__device__ __forceinline__ uint4 pack_c(f32_t, const c2* v) {
  float a, b, c, d;
  split(v[0], a, b);
  split(v[1], c, d);
  return make_uint4(__float_as_uint(a), __float_as_uint(b), __float_as_uint(c), __float_as_uint(d));
}
template <typename St>
__device__ __forceinline__ unsigned pack1(const c2 v) {
  float a, b;
  split(v, a, b);
  if constexpr (std::is_same<St, f16_t>::value) return f2h2(a, b);
  else if constexpr (std::is_same<St, bf16_t>::value) return f2b2(a, b);
  else return f2b2t(a, b);
}
template <typename St>
__device__ __forceinline__ uint4 pack_c(St, const c2* v) {
  return make_uint4(pack1<St>(v[0]), pack1<St>(v[1]), pack1<St>(v[2]), pack1<St>(v[3]));
}
template <typename St>
__device__ __forceinline__ void store_c(uint4* __restrict__ f, size_t site5, size_t n5, const c2* v) {
  constexpr int PC = Store<St>::per_chunk / 2;
#pragma unroll
  for (int c = 0; c < Store<St>::chunks; ++c) f[c * n5 + site5] = pack_c(St{}, v + c * PC);
}

// v <- a v + b P v (P_s, or P_s^dag for DAG; wall factor -m), see apply_lin
template <bool DAG>
__device__ __forceinline__ void lin(c2* v, float a, float b, int s, int Ls, float m) {
  const int up_src = (s + 1) & (Ls - 1), dn_src = (s - 1) & (Ls - 1);
  const float up_f = (s + 1 >= Ls) ? -m : 1.f, dn_f = (s < 1) ? -m : 1.f;
  const int sp = DAG ? up_src : dn_src, sm = DAG ? dn_src : up_src;
  const c2 bp = bc(b * (DAG ? up_f : dn_f)), bm = bc(b * (DAG ? dn_f : up_f)), aa = bc(a);
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = fma(bp, shfl(v[i], sp, Ls), mul(aa, v[i]));
#pragma unroll
  for (int i = 6; i < 12; ++i) v[i] = fma(bm, shfl(v[i], sm, Ls), mul(aa, v[i]));
}

// v <- M_ee^-1 v (DAG: M_ee^-dag) by log2(Ls) doubling steps, see apply_minv
template <bool DAG>
__device__ __forceinline__ void minv(c2* v, int s, const HopArgs& a) {
  const float m = a.fmass;
  const int Ls = a.Ls;
  for (int j = 0; j < a.lslog2; ++j) {
    const int d = 1 << j;
    const int up_src = (s + d) & (Ls - 1), dn_src = (s - d) & (Ls - 1);
    const float up_f = (s + d >= Ls) ? -m : 1.f, dn_f = (s < d) ? -m : 1.f;
    const int sp = DAG ? up_src : dn_src, sm = DAG ? dn_src : up_src;
    const float rp = a.frpow[j];
    const c2 cp = bc(rp * (DAG ? up_f : dn_f)), cm = bc(rp * (DAG ? dn_f : up_f));
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = fma(cp, shfl(v[i], sp, Ls), v[i]);
#pragma unroll
    for (int i = 6; i < 12; ++i) v[i] = fma(cm, shfl(v[i], sm, Ls), v[i]);
  }
  const c2 nrm = bc(a.fminv_norm);
#pragma unroll
  for (int i = 0; i < 12; ++i) v[i] = mul(nrm, v[i]);
}

// h = (1 - SG gamma_MU) psi, upper two spins (see project): per colour c,
//   u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c]
template <int MU, int SG>
__device__ __forceinline__ void proj(const c2* p, c2* h) {
  const c2 pn = make(-(float)SG, (float)SG), np = make((float)SG, -(float)SG);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const c2 u0 = p[c], u1 = p[3 + c], l0 = p[6 + c], l1 = p[9 + c];
    if (MU == 0) {        // h0 = u0 + SG i l1, h1 = u1 + SG i l0
      h[c] = fma(swp(l1), pn, u0);
      h[3 + c] = fma(swp(l0), pn, u1);
    } else if (MU == 1) { // h0 = u0 + SG l1, h1 = u1 - SG l0
      h[c] = SG > 0 ? add(u0, l1) : sub(u0, l1);
      h[3 + c] = SG > 0 ? sub(u1, l0) : add(u1, l0);
    } else if (MU == 2) { // h0 = u0 + SG i l0, h1 = u1 - SG i l1
      h[c] = fma(swp(l0), pn, u0);
      h[3 + c] = fma(swp(l1), np, u1);
    } else {              // h0 = u0 - SG l0, h1 = u1 - SG l1
      h[c] = SG > 0 ? sub(u0, l0) : add(u0, l0);
      h[3 + c] = SG > 0 ? sub(u1, l1) : add(u1, l1);
    }
  }
}

// acc += (uh, -SG B_MU uh) (see reconstruct_add)
template <int MU, int SG>
__device__ __forceinline__ void recon(const c2* uh, c2* acc) {
  const c2 pn = make(-(float)SG, (float)SG), np = make((float)SG, -(float)SG);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const c2 h0 = uh[c], h1 = uh[3 + c];
    acc[c] = add(acc[c], h0);
    acc[3 + c] = add(acc[3 + c], h1);
    if (MU == 0) {        // lower -= SG (i h1, i h0)
      acc[6 + c] = fma(swp(h1), np, acc[6 + c]);
      acc[9 + c] = fma(swp(h0), np, acc[9 + c]);
    } else if (MU == 1) { // lower -= SG (h1, -h0)
      acc[6 + c] = SG > 0 ? sub(acc[6 + c], h1) : add(acc[6 + c], h1);
      acc[9 + c] = SG > 0 ? add(acc[9 + c], h0) : sub(acc[9 + c], h0);
    } else if (MU == 2) { // lower -= SG (i h0, -i h1)
      acc[6 + c] = fma(swp(h0), np, acc[6 + c]);
      acc[9 + c] = fma(swp(h1), pn, acc[9 + c]);
    } else {              // lower -= SG (h0, h1)
      acc[6 + c] = SG > 0 ? sub(acc[6 + c], h0) : add(acc[6 + c], h0);
      acc[9 + c] = SG > 0 ? sub(acc[9 + c], h1) : add(acc[9 + c], h1);
    }
  }
}

// uh[sp][a] = sum_b U[a][b] h[sp][b]; U given as 9 quadruples (u_re, u_re, -u_im, u_im)
__device__ __forceinline__ void su3(const float4* U, const c2* h, c2* uh) {
  c2 sh[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) sh[i] = swp(h[i]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c2 r0 = 0ull, r1 = 0ull;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 q = U[a * 3 + b];
      const c2 P = make(q.x, q.y), Q = make(q.z, q.w);
      if (b == 0) {
        r0 = fma(Q, sh[b], mul(P, h[b]));
        r1 = fma(Q, sh[3 + b], mul(P, h[3 + b]));
      } else {
        r0 = fma(Q, sh[b], fma(P, h[b], r0));
        r1 = fma(Q, sh[3 + b], fma(P, h[3 + b], r1));
      }
    }
    uh[a] = r0;
    uh[3 + a] = r1;
  }
}

// one link's 9 entries from the global link array, expanded to quadruples
template <typename LT>
__device__ __forceinline__ float4 link_entry(const uint4* __restrict__ lk, int e);
template <>
__device__ __forceinline__ float4 link_entry<float2>(const uint4* __restrict__ lk, int e) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(lk) + e);
  return make_float4(v.x, v.x, -v.y, v.y);
}
template <>
__device__ __forceinline__ float4 link_entry<__half2>(const uint4* __restrict__ lk, int e) {
  const float2 v = h2f(__ldg(reinterpret_cast<const unsigned*>(lk) + e));
  return make_float4(v.x, v.x, -v.y, v.y);
}
template <>
__device__ __forceinline__ float4 link_entry<__nv_bfloat162>(const uint4* __restrict__ lk, int e) {
  const float2 v = b2f(__ldg(reinterpret_cast<const unsigned*>(lk) + e));
  return make_float4(v.x, v.x, -v.y, v.y);
}

// link dir of the thread's 4D site: from the staged quadruples, or expanded
// from the global array into registers
template <typename LT, bool STAGE>
__device__ __forceinline__ void su3_dir(const float4* Us, const uint4* lk, int dir, const c2* h, c2* uh) {
  if constexpr (STAGE) {
    su3(Us + dir * 9, h, uh);
  } else {
    constexpr int LG = LinkGran<LT>::g;
    float4 Ul[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) Ul[e] = link_entry<LT>(lk + dir * LG, e);
    su3(Ul, h, uh);
  }
}

// both hops along MU: neighbours x + mu (projector 1 - SF g) and x - mu (1 + SF g)
template <typename St, typename LT, int MU, int SF, bool KIN, bool STAGE>
__device__ __forceinline__ void hop_dir(const HopArgs& a, const uint4* in, const int* nbv, const float4* Us,
                                        const uint4* lk, int s, c2* acc) {
  uint4 gf[Store<St>::chunks], gb[Store<St>::chunks];
  load_raw<St>(in, (size_t)nbv[MU] * a.Ls + s, a.n5, gf);
  load_raw<St>(in, (size_t)nbv[MU + 4] * a.Ls + s, a.n5, gb);
  c2 ps[12], h[6], uh[6];
  unpack_site<St>(gf, ps);
  if (KIN) lin<false>(ps, a.fb, a.fc, s, a.Ls, a.fmass);
  proj<MU, SF>(ps, h);
  su3_dir<LT, STAGE>(Us, lk, MU, h, uh);
  recon<MU, SF>(uh, acc);
  unpack_site<St>(gb, ps);
  if (KIN) lin<false>(ps, a.fb, a.fc, s, a.Ls, a.fmass);
  proj<MU, -SF>(ps, h);
  su3_dir<LT, STAGE>(Us, lk, MU + 4, h, uh);
  recon<MU, -SF>(uh, acc);
}

// |acc|^2 into the FP64 grid reduction (warp sums in double-float, see hop_norm2)
__device__ __forceinline__ void norm2_c(const c2* acc, bool active, const Reduction& red) {
  c2 s2 = 0ull;
  if (active) {
#pragma unroll
    for (int i = 0; i < 12; ++i) s2 = fma(acc[i], acc[i], s2);
  }
  float x, y;
  split(s2, x, y);
  float hi = x, lo = 0.f;
  {
    float sh, eh;
    two_sum(hi, y, sh, eh);
    hi = sh;
    lo = eh;
  }
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
}

// Largest number of 4D sites a CTA of 256 threads covers with staged links (Ls >= 8).
constexpr int PK_SITES = 32;

// One hop pass with packed arithmetic.  STAGE: the CTA's links are staged in
// shared memory (needs Ls >= 8, i.e. at most PK_SITES 4D sites per CTA);
// otherwise every thread expands its site's links itself.
template <typename St, int PASS, bool MOB, int MINB, bool STAGE>
__global__ void __launch_bounds__(256, MINB) hop_packed_kernel(const HopArgs a) {
  using LT = typename LinkOf<St>::T;
  constexpr int LG = LinkGran<LT>::g;
  constexpr bool DAG = (PASS == PASS_C || PASS == PASS_D);
  constexpr int SF = DAG ? -1 : 1;
  __shared__ float4 lsm[STAGE ? PK_SITES : 1][8][9];
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gtid < a.n5;
  const size_t roff = (size_t)blockIdx.y * a.fstride;
  const int rhs = blockIdx.y;
  const int s = threadIdx.x & (a.Ls - 1);
  const size_t x4 = active ? (gtid >> a.lslog2) : 0;
  const size_t site5 = x4 * a.Ls + s;
  const float m = a.fmass;

  const float4* U = nullptr;
  const uint4* lk = reinterpret_cast<const uint4*>(a.links) + x4 * 8 * LG;
  if constexpr (STAGE) {
    const int sites = blockDim.x >> a.lslog2;
    const size_t x40 = ((size_t)blockIdx.x * blockDim.x) >> a.lslog2;
    const uint4* lk0 = reinterpret_cast<const uint4*>(a.links);
    const size_t n4 = a.n5 >> a.lslog2;
    for (int q = threadIdx.x; q < sites * 72; q += blockDim.x) {
      const int ls = q / 72, r = q % 72;
      const size_t xs = x40 + ls;
      lsm[ls][r / 9][r % 9] = xs < n4 ? link_entry<LT>(lk0 + (xs * 8 + r / 9) * LG, r % 9)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    U = &lsm[threadIdx.x >> a.lslog2][0][0];
  }

  c2 acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = 0ull;
  const uint4* in = a.in + roff;
  const int4 nb0 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2);
  const int4 nb1 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2 + 1);
  const int nbv[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};
  constexpr bool KIN = PASS == PASS_A && MOB;
  hop_dir<St, LT, 0, SF, KIN, STAGE>(a, in, nbv, U, lk, s, acc);
  hop_dir<St, LT, 1, SF, KIN, STAGE>(a, in, nbv, U, lk, s, acc);
  hop_dir<St, LT, 2, SF, KIN, STAGE>(a, in, nbv, U, lk, s, acc);
  hop_dir<St, LT, 3, SF, KIN, STAGE>(a, in, nbv, U, lk, s, acc);

  if (PASS == PASS_A) {
    minv<false>(acc, s, a);
    if (MOB) {
      lin<false>(acc, a.fb, a.fc, s, a.Ls, m);
    } else {
      const c2 bb = bc(a.fb * a.fb);
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = mul(bb, acc[i]);
    }
  } else if (PASS == PASS_C) {
    if (MOB) {
      lin<true>(acc, a.fb, a.fc, s, a.Ls, m);
    } else {
      const c2 bb = bc(a.fb);
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = mul(bb, acc[i]);
    }
    minv<true>(acc, s, a);
  } else {
    // B, D: out = M_oo^(dag) in2 - K^(dag) acc / 4   (B has no K on this side)
    if (PASS == PASS_D) {
      if (MOB) {
        lin<true>(acc, a.fb, a.fc, s, a.Ls, m);
      } else {
        const c2 bb = bc(a.fb);
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = mul(bb, acc[i]);
      }
    }
    c2 self[12];
    load_c<St>(a.in2 + roff, site5, a.n5, self);
    lin<DAG>(self, a.falpha, a.fbeta, s, a.Ls, m);
    const c2 q = bc(-0.25f);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = fma(q, acc[i], self[i]);
    if (PASS == PASS_D) {
      const c2 sD = bc(a.fsD);
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = mul(sD, acc[i]);
      if (a.extra) {
        c2 ex[12];
        load_c<St>(a.extra + roff, site5, a.n5, ex);
        const c2 lam = bc(a.flam);
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = fma(lam, ex[i], acc[i]);
      }
    }
  }
  if (PASS == PASS_D && a.cg_r) {
    __shared__ float s_alpha;
    if (threadIdx.x == 0) {
      double den = a.al_den0[rhs];
      if (a.al_den1) den += a.al_lam * a.al_den1[rhs];
      const bool live = a.al_mask == nullptr || a.al_mask[rhs] != 0;
      s_alpha = (float)((den != 0.0 && live) ? a.al_num[rhs] / den : 0.0);
    }
    __syncthreads();
    if (active) {
      const c2 al = bc(s_alpha), nal = bc(-s_alpha);
      c2 rv[12], xv[12], pv[12];
      load_c<St>(a.cg_r + roff, site5, a.n5, rv);
      load_c<St>(a.cg_x + roff, site5, a.n5, xv);
      load_c<St>(a.cg_p + roff, site5, a.n5, pv);
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        rv[i] = fma(nal, acc[i], rv[i]);
        xv[i] = fma(al, pv[i], xv[i]);
        acc[i] = rv[i];
      }
      store_c<St>(a.cg_r + roff, site5, a.n5, rv);
      store_c<St>(a.cg_x + roff, site5, a.n5, xv);
    }
  } else if (active) {
    store_c<St>(a.out + roff, site5, a.n5, acc);
  }
  if (a.do_red) norm2_c(acc, active, a.red);
}

}  // namespace pk
}  // namespace hdcg
