// Reduced-precision spinor codecs of Sec. 6.5 ("Reduced precision in
// preconditioner communication", Table sloppy).
//
// 8-bit format: one 5D site's 24 reals as a half-precision prefactor and 24
// signed bytes.  The prefactor is the largest |real| of the site rounded to
// FP16 (round to nearest even); each real becomes round(127 v / prefactor)
// (ties to even) clipped to [-127, 127]; decoding multiplies by prefactor / 127.
// 26 bytes per site against 48 (FP16) and 96 (FP32).  The canonical entry
// points work in FP64 on complex double fields (bit-for-bit the definition);
// the solver's round trip (sloppy_codec) works in FP32 on the internal field.
// The 16-bit format is the truncation of each FP32 word to its top 16 bits
// (HDCG_BF16T storage).
#include "blas.cuh"

namespace hdcg {

namespace {

__global__ void k_encode_i8(const double* __restrict__ in, __half* scale, int8_t* q, size_t n5) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const double* v = in + t * 24;
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 24; ++i) s = fmax(s, fabs(v[i]));
  const __half sh = __double2half(s);
  const double sf = (double)__half2float(sh);
  scale[t] = sh;
#pragma unroll
  for (int i = 0; i < 24; ++i) {
    double r = sf > 0.0 ? rint(127.0 * v[i] / sf) : 0.0;
    r = fmin(127.0, fmax(-127.0, r));
    q[t * 24 + i] = (int8_t)(int)r;
  }
}

__global__ void k_decode_i8(const __half* __restrict__ scale, const int8_t* __restrict__ q, double* out, size_t n5) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const double f = (double)__half2float(scale[t]) / 127.0;
#pragma unroll
  for (int i = 0; i < 24; ++i) out[t * 24 + i] = (double)q[t * 24 + i] * f;
}

// in place: v <- decode(encode(v)) per 5D site, FP32 arithmetic (codec 2), or
// each float32 word truncated to its top 16 bits (codec 1)
template <typename St>
__global__ void k_codec_roundtrip(uint4* f, size_t n5, size_t fstride, int codec) {
  using R = typename Store<St>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  uint4* g = f + blockIdx.y * fstride;
  R v[24];
  load_spinor<St, R>(g, t, n5, v);
  if (codec == 1) {
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(__float_as_uint((float)v[i]) & 0xffff0000u);
  } else {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 24; ++i) s = fmaxf(s, fabsf((float)v[i]));
    const float sf = __half2float(__float2half_rn(s));
    const float k = sf > 0.f ? 127.f / sf : 0.f, f = sf / 127.f;
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = fminf(127.f, fmaxf(-127.f, rintf((float)v[i] * k))) * f;
  }
  store_spinor<St, R>(g, t, n5, v);
}

}  // namespace

void encode_i8(Ctx& c, const void* in, void* scale, void* q, size_t nfields) {
  const size_t n = c.n5 * nfields;
  k_encode_i8<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>((const double*)in, (__half*)scale, (int8_t*)q, n);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void decode_i8(Ctx& c, const void* scale, const void* q, void* out, size_t nfields) {
  const size_t n = c.n5 * nfields;
  k_decode_i8<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>((const __half*)scale, (const int8_t*)q, (double*)out,
                                                                 n);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void codec_roundtrip(Ctx& c, uint4* f, int prec, int codec, int nrhs) {
  if (codec == 0) return;
  HDCG_REQUIRE(codec == 1 || codec == 2, HDCG_ERR_ARG, "sloppy_codec must be 0, 1 or 2");
  const dim3 grid((unsigned)((c.n5 + 255) / 256), (unsigned)nrhs);
  const size_t fs = c.field_bytes(prec) / 16;
  DISPATCH_PREC(prec, S, { k_codec_roundtrip<S><<<grid, 256, 0, c.stream>>>(f, c.n5, fs, codec); });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

}  // namespace hdcg
