// Field conversions and BLAS-1 kernels of the HDCG library.
//
// All kernels run one thread per 5D site and move the site's 24 reals with
// load_spinor / store_spinor, so operands of different storage precision (and
// hence different chunking) line up.  Every reduction accumulates in FP64
// (per-thread FP32/FP64 partial over 24 reals, then FP64 warp / block / grid
// sums in a fixed order: two runs give bit-identical results).
#include "blas.cuh"

namespace hdcg {

// ---------------------------------------------------------------------------
// canonical <-> internal
// ---------------------------------------------------------------------------
template <typename CT> struct Canon;
template <> struct Canon<f64_t> {
  static __device__ __forceinline__ double ld(const void* p, size_t i) { return ((const double*)p)[i]; }
  static __device__ __forceinline__ void st(void* p, size_t i, double v) { ((double*)p)[i] = v; }
};
template <> struct Canon<f32_t> {
  static __device__ __forceinline__ double ld(const void* p, size_t i) { return ((const float*)p)[i]; }
  static __device__ __forceinline__ void st(void* p, size_t i, double v) { ((float*)p)[i] = (float)v; }
};
template <> struct Canon<f16_t> {
  static __device__ __forceinline__ double ld(const void* p, size_t i) {
    return __half2float(((const __half*)p)[i]);
  }
  static __device__ __forceinline__ void st(void* p, size_t i, double v) {
    ((__half*)p)[i] = __float2half_rn((float)v);
  }
};
template <> struct Canon<bf16_t> {
  static __device__ __forceinline__ double ld(const void* p, size_t i) {
    return __bfloat162float(((const __nv_bfloat16*)p)[i]);
  }
  static __device__ __forceinline__ void st(void* p, size_t i, double v) {
    ((__nv_bfloat16*)p)[i] = __float2bfloat16_rn((float)v);
  }
};
template <> struct Canon<bf16t_t> {
  static __device__ __forceinline__ double ld(const void* p, size_t i) {
    return __bfloat162float(((const __nv_bfloat16*)p)[i]);
  }
  static __device__ __forceinline__ void st(void* p, size_t i, double v) {
    unsigned u = __float_as_uint((float)v) >> 16;
    ((unsigned short*)p)[i] = (unsigned short)u;
  }
};

template <typename CT, typename So>
__global__ void k_canon_to_int(const void* __restrict__ canon, uint4* __restrict__ out, size_t n5,
                               size_t nf) {
  using R = typename Store<So>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5 * nf) return;
  const size_t f = t / n5, site5 = t % n5;
  R v[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] = (R)Canon<CT>::ld(canon, t * 24 + i);
  store_spinor<So, R>(out + f * n5 * Store<So>::chunks, site5, n5, v);
}

template <typename Si, typename CT>
__global__ void k_int_to_canon(const uint4* __restrict__ in, void* __restrict__ canon, size_t n5,
                               size_t nf) {
  using R = typename Store<Si>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5 * nf) return;
  const size_t f = t / n5, site5 = t % n5;
  R v[24];
  load_spinor<Si, R>(in + f * n5 * Store<Si>::chunks, site5, n5, v);
#pragma unroll
  for (int i = 0; i < 24; ++i) Canon<CT>::st(canon, t * 24 + i, (double)v[i]);
}

template <typename Si, typename So>
__global__ void k_convert(const uint4* __restrict__ in, uint4* __restrict__ out, size_t n5, size_t nf) {
  using Ri = typename Store<Si>::real;
  using Ro = typename Store<So>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5 * nf) return;
  const size_t f = t / n5, site5 = t % n5;
  Ri v[24];
  load_spinor<Si, Ri>(in + f * n5 * Store<Si>::chunks, site5, n5, v);
  Ro w[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) w[i] = (Ro)v[i];
  store_spinor<So, Ro>(out + f * n5 * Store<So>::chunks, site5, n5, w);
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256); }

void canon_to_internal(Ctx& c, const void* canon, int canon_prec, uint4* out, int prec, size_t nf) {
  const unsigned g = blocks_for(c.n5 * nf);
  if (prec == HDCG_DF64 || canon_prec == HDCG_DF64) {   // complex double canonical <-> double-float
    HDCG_REQUIRE(prec == HDCG_DF64 && (canon_prec == HDCG_F64 || canon_prec == HDCG_DF64), HDCG_ERR_ARG,
                 "double-float fields convert from complex double only");
    k_canon_to_int<f64_t, df_t><<<g, 256, 0, c.stream>>>(canon, out, c.n5, nf);
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
    return;
  }
  DISPATCH_PREC(canon_prec, CT, {
    DISPATCH_PREC(prec, So, { k_canon_to_int<CT, So><<<g, 256, 0, c.stream>>>(canon, out, c.n5, nf); });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void internal_to_canon(Ctx& c, const uint4* in, int prec, void* canon, int canon_prec, size_t nf) {
  const unsigned g = blocks_for(c.n5 * nf);
  if (prec == HDCG_DF64 || canon_prec == HDCG_DF64) {
    HDCG_REQUIRE(prec == HDCG_DF64 && (canon_prec == HDCG_F64 || canon_prec == HDCG_DF64), HDCG_ERR_ARG,
                 "double-float fields convert to complex double only");
    k_int_to_canon<df_t, f64_t><<<g, 256, 0, c.stream>>>(in, canon, c.n5, nf);
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
    return;
  }
  DISPATCH_PREC(prec, Si, {
    DISPATCH_PREC(canon_prec, CT, { k_int_to_canon<Si, CT><<<g, 256, 0, c.stream>>>(in, canon, c.n5, nf); });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void convert_field(Ctx& c, const uint4* in, int pin, uint4* out, int pout, size_t nf) {
  const unsigned g = blocks_for(c.n5 * nf);
  if (pin == HDCG_DF64 || pout == HDCG_DF64) {   // FP64 <-> double-float only
    if (pin == HDCG_F64 && pout == HDCG_DF64) k_convert<f64_t, df_t><<<g, 256, 0, c.stream>>>(in, out, c.n5, nf);
    else if (pin == HDCG_DF64 && pout == HDCG_F64) k_convert<df_t, f64_t><<<g, 256, 0, c.stream>>>(in, out, c.n5, nf);
    else throw Error{HDCG_ERR_ARG, "double-float fields convert to and from FP64 only"};
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
    return;
  }
  DISPATCH_PREC(pin, Si, {
    DISPATCH_PREC(pout, So, { k_convert<Si, So><<<g, 256, 0, c.stream>>>(in, out, c.n5, nf); });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void zero_field(Ctx& c, uint4* f, int prec, size_t nf) {
  HDCG_CUDA(cudaMemsetAsync(f, 0, c.field_bytes(prec) * nf, c.stream));
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_norm2(const uint4* __restrict__ a, size_t n5, Reduction red, size_t fstride) {
  using R = typename Store<S>::real;
  a += blockIdx.y * fstride;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < n5) {
    R x[24];
    load_spinor<S, R>(a, t, n5, x);
    R s = 0;
#pragma unroll
    for (int i = 0; i < 24; ++i) s += x[i] * x[i];
    v[0] = (double)s;
  }
  grid_reduce<1>(v, red);
}

template <typename S>
__global__ void k_cdot(const uint4* __restrict__ a, const uint4* __restrict__ b, size_t n5, Reduction red) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (t < n5) {
    R x[24], y[24];
    load_spinor<S, R>(a, t, n5, x);
    load_spinor<S, R>(b, t, n5, y);
    R re = 0, im = 0;
#pragma unroll
    for (int i = 0; i < 24; i += 2) {
      re += x[i] * y[i] + x[i + 1] * y[i + 1];
      im += x[i] * y[i + 1] - x[i + 1] * y[i];
    }
    v[0] = (double)re;
    v[1] = (double)im;
  }
  grid_reduce<2>(v, red);
}

Reduction make_reduction(Ctx& c, unsigned grid, int nv, double* result, int accumulate, int nrhs) {
  c.red_partials.ensure((size_t)grid * nv * nrhs * sizeof(double) + 64);
  Reduction r;
  r.partials = c.red_partials.as<double>();
  r.ticket = c.red_ticket.as<unsigned>();
  r.result = result;
  r.accumulate = accumulate;
  r.result_stride = nv;  // NV values per right-hand side, contiguous
  return r;
}

void norm2(Ctx& c, const uint4* a, int prec, size_t /*n_reals*/, double* result, int nrhs) {
  const unsigned g = blocks_for(c.n5);
  Reduction r = make_reduction(c, g, 1, result, 0, nrhs);
  const size_t fs = c.field_bytes(prec) / 16;
  DISPATCH_PREC(prec, S, { k_norm2<S><<<dim3(g, nrhs), 256, 0, c.stream>>>(a, c.n5, r, fs); });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void cdot(Ctx& c, const uint4* a, const uint4* b, int prec, size_t /*n_reals*/, double* result) {
  const unsigned g = blocks_for(c.n5);
  Reduction r = make_reduction(c, g, 2, result, 0);
  DISPATCH_PREC(prec, S, { k_cdot<S><<<g, 256, 0, c.stream>>>(a, b, c.n5, r); });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// ---------------------------------------------------------------------------
// Krylov updates.  Scalars are read from device memory (no host round trip):
//   alpha = num / (den0 + lam * den1)      (den1 may be null)
//   beta  = (n0 - n1) / d                  (n1 may be null)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ratio(const double* num, const double* den0, const double* den1,
                                        double lam) {
  double d = *den0;
  if (den1) d += lam * (*den1);
  return d != 0.0 ? *num / d : 0.0;
}

// x += alpha p ; r -= alpha w ; |r|^2 -> red   (x may have its own precision)
template <typename Sx, typename S>
__global__ void k_update_xr(uint4* x, const uint4* __restrict__ p, uint4* r, const uint4* __restrict__ w,
                            size_t n5, ScalarRef al, int sign_x, Reduction red) {
  using Rx = typename Store<Sx>::real;
  using R = typename Store<S>::real;
  const double alpha = ratio(al.num, al.den0, al.den1, al.lam);
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < n5) {
    R pv[24], rv[24], wv[24];
    Rx xv[24];
    load_spinor<S, R>(p, t, n5, pv);
    load_spinor<S, R>(r, t, n5, rv);
    load_spinor<S, R>(w, t, n5, wv);
    if (x) load_spinor<Sx, Rx>(x, t, n5, xv);
    const R a = (R)alpha;
    const Rx ax = (Rx)(sign_x * alpha);
    R s = 0;
#pragma unroll
    for (int i = 0; i < 24; ++i) {
      if (x) xv[i] += ax * (Rx)pv[i];
      rv[i] -= a * wv[i];
      s += rv[i] * rv[i];
    }
    if (x) store_spinor<Sx, Rx>(x, t, n5, xv);
    store_spinor<S, R>(r, t, n5, rv);
    v[0] = (double)s;
  }
  grid_reduce<1>(v, red);
}

// p = y + beta p ; optional |p|^2 -> red
template <typename S>
__global__ void k_update_p(uint4* p, const uint4* __restrict__ y, size_t n5, ScalarRef be, int do_red,
                           Reduction red, size_t fstride) {
  using R = typename Store<S>::real;
  const int rr = blockIdx.y;
  p += rr * fstride;
  y += rr * fstride;
  double beta = 0.0;
  {
    double n = be.num[rr * be.stride];
    if (be.den1) n -= be.den1[rr * be.stride];  // n1 stored in den1 slot for beta
    const double d = be.den0[rr];
    beta = d != 0.0 ? n / d : 0.0;
  }
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < n5) {
    R pv[24], yv[24];
    load_spinor<S, R>(p, t, n5, pv);
    load_spinor<S, R>(y, t, n5, yv);
    R s = 0;
    const R b = (R)beta;
#pragma unroll
    for (int i = 0; i < 24; ++i) {
      pv[i] = yv[i] + b * pv[i];
      s += pv[i] * pv[i];
    }
    store_spinor<S, R>(p, t, n5, pv);
    v[0] = (double)s;
  }
  if (do_red) grid_reduce<1>(v, red);
}

// res[0] = Re<a, b>, res[1] = Re<a, c> (c may be null)
template <typename S>
__global__ void k_redot2(const uint4* __restrict__ a, const uint4* __restrict__ b, const uint4* __restrict__ cc,
                         size_t n5, Reduction red, size_t fstride) {
  using R = typename Store<S>::real;
  const size_t ro = blockIdx.y * fstride;
  a += ro;
  b += ro;
  if (cc) cc += ro;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (t < n5) {
    R av[24], bv[24];
    load_spinor<S, R>(a, t, n5, av);
    load_spinor<S, R>(b, t, n5, bv);
    R s0 = 0, s1 = 0;
#pragma unroll
    for (int i = 0; i < 24; ++i) s0 += av[i] * bv[i];
    if (cc) {
      R cv[24];
      load_spinor<S, R>(cc, t, n5, cv);
#pragma unroll
      for (int i = 0; i < 24; ++i) s1 += av[i] * cv[i];
    }
    v[0] = (double)s0;
    v[1] = (double)s1;
  }
  grid_reduce<2>(v, red);
}

// hi += lo ; lo = 0
template <typename Sh, typename Sl>
__global__ void k_accum_hi(uint4* hi, uint4* lo, size_t n5, size_t fsh, size_t fsl) {
  using Rh = typename Store<Sh>::real;
  using Rl = typename Store<Sl>::real;
  hi += blockIdx.y * fsh;
  lo += blockIdx.y * fsl;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  Rh h[24];
  Rl l[24];
  load_spinor<Sh, Rh>(hi, t, n5, h);
  load_spinor<Sl, Rl>(lo, t, n5, l);
#pragma unroll
  for (int i = 0; i < 24; ++i) {
    h[i] += (Rh)l[i];
    l[i] = 0;
  }
  store_spinor<Sh, Rh>(hi, t, n5, h);
  store_spinor<Sl, Rl>(lo, t, n5, l);
}

// y = a x + b y (host scalars); x may have another precision than y
template <typename Sx, typename Sy>
__global__ void k_axpby(double a, const uint4* __restrict__ x, double b, uint4* y, size_t n5) {
  using Rx = typename Store<Sx>::real;
  using Ry = typename Store<Sy>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  Rx xv[24];
  Ry yv[24];
  load_spinor<Sx, Rx>(x, t, n5, xv);
  if (b != 0.0) load_spinor<Sy, Ry>(y, t, n5, yv);
#pragma unroll
  for (int i = 0; i < 24; ++i) yv[i] = (Ry)a * (Ry)xv[i] + (b != 0.0 ? (Ry)b * yv[i] : Ry(0));
  store_spinor<Sy, Ry>(y, t, n5, yv);
}

// y = scale * x with scale = sqrt(num / den) read on the device (normalisation)
template <typename S>
__global__ void k_scale_dev(const uint4* __restrict__ x, uint4* y, size_t n5, const double* num,
                            const double* den, int inv) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  double q = *den > 0 ? *num / *den : 0.0;
  double s = sqrt(q);
  if (inv) s = s > 0 ? 1.0 / s : 0.0;
  R v[24];
  load_spinor<S, R>(x, t, n5, v);
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] *= (R)s;
  store_spinor<S, R>(y, t, n5, v);
}

// out = s * in with s = sqrt(num / den) (inv: 1 / s), precisions may differ
template <typename Si, typename So>
__global__ void k_convert_scaled(const uint4* __restrict__ in, uint4* __restrict__ out, size_t n5,
                                 const double* num, const double* den, int inv, size_t fsi, size_t fso) {
  using Ri = typename Store<Si>::real;
  using Ro = typename Store<So>::real;
  const int rr = blockIdx.y;
  in += rr * fsi;
  out += rr * fso;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const double nv = num[0], dv = den[rr];
  const double q = (dv > 0.0 && nv > 0.0) ? nv / dv : 1.0;
  double sc = sqrt(q);
  if (inv) sc = 1.0 / sc;
  Ri v[24];
  load_spinor<Si, Ri>(in, t, n5, v);
  Ro w[24];
  const Ro s = (Ro)sc;
#pragma unroll
  for (int i = 0; i < 24; ++i) w[i] = (Ro)v[i] * s;
  store_spinor<So, Ro>(out, t, n5, w);
}

void convert_scaled(Ctx& c, const uint4* in, int pin, uint4* out, int pout, const double* num, const double* den,
                    int inv, int nrhs) {
  const unsigned g = blocks_for(c.n5);
  const size_t fsi = c.field_bytes(pin) / 16, fso = c.field_bytes(pout) / 16;
  DISPATCH_PREC(pin, Si, {
    DISPATCH_PREC(pout, So, {
      k_convert_scaled<Si, So><<<dim3(g, nrhs), 256, 0, c.stream>>>(in, out, c.n5, num, den, inv, fsi, fso);
    });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// amax[r] = max |real| of field r (as float bits: non-negative floats order like
// their bit patterns)
template <typename S>
__global__ void k_amax(const uint4* __restrict__ x, size_t n5, size_t fs, unsigned* amax) {
  using R = typename Store<S>::real;
  const int rr = blockIdx.y;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.f;
  if (t < n5) {
    R v[24];
    load_spinor<S, R>(x + rr * fs, t, n5, v);
#pragma unroll
    for (int i = 0; i < 24; ++i) m = fmaxf(m, fabsf((float)v[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(amax + rr, __float_as_uint(m));
}

__global__ void k_cap_den(const unsigned* amax, const double* num, double* den, double peak, int nrhs) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  const double m = (double)__uint_as_float(amax[r]) / peak;
  const double d = num[0] * m * m;
  if (d > den[r]) den[r] = d;
}

void cap_scale(Ctx& c, const uint4* x, int prec, const double* num, double* den, double peak, unsigned* amax,
               int nrhs) {
  HDCG_CUDA(cudaMemsetAsync(amax, 0, nrhs * sizeof(unsigned), c.stream));
  const size_t fs = c.field_bytes(prec) / 16;
  DISPATCH_PREC(prec, S, { k_amax<S><<<dim3(blocks_for(c.n5), nrhs), 256, 0, c.stream>>>(x, c.n5, fs, amax); });
  k_cap_den<<<1, 32, 0, c.stream>>>(amax, num, den, peak, nrhs);
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2;
}

void update_xr(Ctx& c, int prec_x, uint4* x, int prec, const uint4* p, uint4* r, const uint4* w,
               ScalarRef alpha, int sign_x, double* rr_out) {
  const unsigned g = blocks_for(c.n5);
  Reduction red = make_reduction(c, g, 1, rr_out, 0);
  DISPATCH_PREC(prec_x, Sx, {
    DISPATCH_PREC(prec, S, { k_update_xr<Sx, S><<<g, 256, 0, c.stream>>>(x, p, r, w, c.n5, alpha, sign_x, red); });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void update_p(Ctx& c, int prec, uint4* p, const uint4* y, ScalarRef beta, double* pp_out, int nrhs) {
  const unsigned g = blocks_for(c.n5);
  Reduction red = make_reduction(c, g, 1, pp_out, 0, nrhs);
  const size_t fs = c.field_bytes(prec) / 16;
  DISPATCH_PREC(prec, S, {
    k_update_p<S><<<dim3(g, nrhs), 256, 0, c.stream>>>(p, y, c.n5, beta, pp_out != nullptr, red, fs);
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void redot2(Ctx& c, int prec, const uint4* a, const uint4* b, const uint4* cc, double* out2, int nrhs) {
  const unsigned g = blocks_for(c.n5);
  Reduction red = make_reduction(c, g, 2, out2, 0, nrhs);
  const size_t fs = c.field_bytes(prec) / 16;
  DISPATCH_PREC(prec, S, { k_redot2<S><<<dim3(g, nrhs), 256, 0, c.stream>>>(a, b, cc, c.n5, red, fs); });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void accum_hi(Ctx& c, int prec_hi, uint4* hi, int prec_lo, uint4* lo, int nrhs) {
  const unsigned g = blocks_for(c.n5);
  const size_t fsh = c.field_bytes(prec_hi) / 16, fsl = c.field_bytes(prec_lo) / 16;
  DISPATCH_PREC(prec_hi, Sh, {
    DISPATCH_PREC(prec_lo, Sl, {
      k_accum_hi<Sh, Sl><<<dim3(g, nrhs), 256, 0, c.stream>>>(hi, lo, c.n5, fsh, fsl);
    });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void axpby(Ctx& c, double a, int prec_x, const uint4* x, double b, int prec_y, uint4* y) {
  const unsigned g = blocks_for(c.n5);
  DISPATCH_PREC(prec_x, Sx, {
    DISPATCH_PREC(prec_y, Sy, { k_axpby<Sx, Sy><<<g, 256, 0, c.stream>>>(a, x, b, y, c.n5); });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void scale_dev(Ctx& c, int prec, const uint4* x, uint4* y, const double* num, const double* den, int inv) {
  const unsigned g = blocks_for(c.n5);
  DISPATCH_PREC(prec, S, { k_scale_dev<S><<<g, 256, 0, c.stream>>>(x, y, c.n5, num, den, inv); });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

}  // namespace hdcg
