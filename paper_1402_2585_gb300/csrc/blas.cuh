// Declarations shared by the library's translation units: precision dispatch,
// device-scalar references and the BLAS-1 entry points (blas.cu).
#pragma once

#include "common.cuh"
#include "context.h"

namespace hdcg {

static_assert(RMAX == RED_RHS, "reduction groups hold one slot per right-hand side");


// Run `body` with `T` bound to the storage tag of precision code `prec`.
#define DISPATCH_PREC(prec, T, ...)                                   \
  switch (prec) {                                                     \
    case HDCG_F64: { using T = f64_t; __VA_ARGS__; } break;           \
    case HDCG_F32: { using T = f32_t; __VA_ARGS__; } break;           \
    case HDCG_F16: { using T = f16_t; __VA_ARGS__; } break;           \
    case HDCG_BF16: { using T = bf16_t; __VA_ARGS__; } break;         \
    case HDCG_BF16T: { using T = bf16t_t; __VA_ARGS__; } break;       \
    default: throw Error{HDCG_ERR_ARG, "unknown precision code"};     \
  }

// Subspace storage precisions (F64, F32, F16) and assembly precisions (F64, F32).
#define DISPATCH_SUB(prec, T, ...)                                     \
  switch (prec) {                                                     \
    case HDCG_F64: { using T = f64_t; __VA_ARGS__; } break;           \
    case HDCG_F32: { using T = f32_t; __VA_ARGS__; } break;           \
    case HDCG_F16: { using T = f16_t; __VA_ARGS__; } break;           \
    default: throw Error{HDCG_ERR_ARG, "unsupported subspace precision"}; \
  }
#define DISPATCH_HI(prec, T, ...)                                      \
  switch (prec) {                                                     \
    case HDCG_F64: { using T = f64_t; __VA_ARGS__; } break;           \
    case HDCG_F32: { using T = f32_t; __VA_ARGS__; } break;           \
    default: throw Error{HDCG_ERR_ARG, "unsupported precision"};      \
  }

// A scalar computed on the device from device doubles:
//   alpha = num / (den0 + lam * den1)   or   beta = (num - den1) / den0
struct ScalarRef {
  const double* num = nullptr;
  const double* den0 = nullptr;
  const double* den1 = nullptr;
  double lam = 0.0;
  int stride = 1;  // right-hand side r reads ptr[r * stride]
};

// Reduction of NV values per block (nrhs right-hand sides along grid y); the
// results of right-hand side r are result[r * nv + i].
Reduction make_reduction(Ctx& c, unsigned grid, int nv, double* result, int accumulate, int nrhs = 1);

// x += sign_x * alpha p (x may be null); r -= alpha w; rr_out = |r|^2
void update_xr(Ctx& c, int prec_x, uint4* x, int prec, const uint4* p, uint4* r, const uint4* w,
               ScalarRef alpha, int sign_x, double* rr_out);
// p = y + beta p; pp_out (may be null) = |p|^2
void update_p(Ctx& c, int prec, uint4* p, const uint4* y, ScalarRef beta, double* pp_out, int nrhs = 1);
// out2[0] = Re<a, b>, out2[1] = Re<a, cc> (cc may be null)
void redot2(Ctx& c, int prec, const uint4* a, const uint4* b, const uint4* cc, double* out2, int nrhs = 1);
// hi += lo; lo = 0
void accum_hi(Ctx& c, int prec_hi, uint4* hi, int prec_lo, uint4* lo, int nrhs = 1);
// y = a x + b y
void axpby(Ctx& c, double a, int prec_x, const uint4* x, double b, int prec_y, uint4* y);
// out = sqrt(num / den)^(inv ? -1 : 1) in, converting precision
// (den is read per right-hand side: den[r]; num[0] is shared)
void convert_scaled(Ctx& c, const uint4* in, int pin, uint4* out, int pout, const double* num, const double* den,
                    int inv, int nrhs = 1);
// den[r] = max(den[r], num[0] (amax_r / peak)^2), amax_r the largest |real| of
// field r of x: the scale sqrt(num / den) then also keeps every real of the
// scaled field within peak (amax: device scratch of nrhs unsigned)
void cap_scale(Ctx& c, const uint4* x, int prec, const double* num, double* den, double peak, unsigned* amax,
               int nrhs = 1);
// y = sqrt(num/den)^(inv ? -1 : 1) x
void scale_dev(Ctx& c, int prec, const uint4* x, uint4* y, const double* num, const double* den, int inv);

// reduced-precision codecs of Sec. 6.5 (codec.cu): canonical complex double
// fields <-> (FP16 prefactor per 5D site, 24 int8 per site); and the solver's
// in-place round trip of an internal field (codec 1: 16-bit truncation, 2: 8-bit)
void encode_i8(Ctx& c, const void* in, void* scale, void* q, size_t nfields);
void decode_i8(Ctx& c, const void* scale, const void* q, void* out, size_t nfields);
void codec_roundtrip(Ctx& c, uint4* f, int prec, int codec, int nrhs = 1);

}  // namespace hdcg
