// Common device helpers of the HDCG library: storage codecs for the internal
// chunked field layout and deterministic FP64 reductions.
//
// Internal fine-field layout ("chunked"): the 24 reals of one 5D site
// (site5 = cb4 * Ls + s; reals ordered [spin][colour][re, im]) are split into
// 16-byte chunks, and chunk c of every site is stored contiguously:
//   field[c * n5 + site5]  (uint4 granules).
// FP64: 12 chunks of 2 doubles, FP32: 6 chunks of 4 floats, 16-bit: 3 chunks
// of 8 halves.  Consecutive threads (consecutive s, then sites) therefore
// load consecutive 16-byte granules.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace hdcg {

constexpr unsigned FULL_MASK = 0xffffffffu;

// storage tags -------------------------------------------------------------
struct f64_t {};
struct f32_t {};
struct f16_t {};
struct bf16_t {};
struct bf16t_t {};  // bfloat16 by truncation of the float32 word
struct df_t {};     // double-float: (hi, lo) float32 pairs

template <typename St> struct Store;
template <> struct Store<f64_t> {
  using real = double;
  static constexpr int per_chunk = 2;
  static constexpr int chunks = 12;
  static constexpr int bytes_per_real = 8;
};
template <> struct Store<f32_t> {
  using real = float;
  static constexpr int per_chunk = 4;
  static constexpr int chunks = 6;
  static constexpr int bytes_per_real = 4;
};
template <> struct Store<f16_t> {
  using real = float;
  static constexpr int per_chunk = 8;
  static constexpr int chunks = 3;
  static constexpr int bytes_per_real = 2;
};
template <> struct Store<df_t> {
  using real = dfl;
  static constexpr int per_chunk = 2;
  static constexpr int chunks = 12;
  static constexpr int bytes_per_real = 8;
};
template <> struct Store<bf16_t> : Store<f16_t> {};
template <> struct Store<bf16t_t> : Store<f16_t> {};

// unpack one 16-byte granule into per_chunk reals ----------------------------
__device__ __forceinline__ void unpack(f64_t, const uint4& g, double* r) {
  r[0] = __hiloint2double(g.y, g.x);
  r[1] = __hiloint2double(g.w, g.z);
}
__device__ __forceinline__ void unpack(f32_t, const uint4& g, float* r) {
  r[0] = __uint_as_float(g.x);
  r[1] = __uint_as_float(g.y);
  r[2] = __uint_as_float(g.z);
  r[3] = __uint_as_float(g.w);
}
__device__ __forceinline__ float2 h2f(unsigned v) {
  __half2 h = *reinterpret_cast<__half2*>(&v);
  return __half22float2(h);
}
__device__ __forceinline__ float2 b2f(unsigned v) {
  // bfloat16 -> float is a 16-bit shift
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}
__device__ __forceinline__ void unpack(f16_t, const uint4& g, float* r) {
  float2 a = h2f(g.x), b = h2f(g.y), c = h2f(g.z), d = h2f(g.w);
  r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  r[4] = c.x; r[5] = c.y; r[6] = d.x; r[7] = d.y;
}
__device__ __forceinline__ void unpack(bf16_t, const uint4& g, float* r) {
  float2 a = b2f(g.x), b = b2f(g.y), c = b2f(g.z), d = b2f(g.w);
  r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  r[4] = c.x; r[5] = c.y; r[6] = d.x; r[7] = d.y;
}
__device__ __forceinline__ void unpack(bf16t_t, const uint4& g, float* r) { unpack(bf16_t{}, g, r); }
__device__ __forceinline__ void unpack(df_t, const uint4& g, dfl* r) {
  r[0] = dfl(__uint_as_float(g.x), __uint_as_float(g.y));
  r[1] = dfl(__uint_as_float(g.z), __uint_as_float(g.w));
}

// pack per_chunk reals into one granule ---------------------------------------
__device__ __forceinline__ uint4 pack(f64_t, const double* r) {
  uint4 g;
  g.x = __double2loint(r[0]); g.y = __double2hiint(r[0]);
  g.z = __double2loint(r[1]); g.w = __double2hiint(r[1]);
  return g;
}
__device__ __forceinline__ uint4 pack(f32_t, const float* r) {
  return make_uint4(__float_as_uint(r[0]), __float_as_uint(r[1]), __float_as_uint(r[2]),
                    __float_as_uint(r[3]));
}
__device__ __forceinline__ unsigned f2h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<unsigned*>(&h);
}
__device__ __forceinline__ unsigned f2b2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<unsigned*>(&h);
}
__device__ __forceinline__ unsigned f2b2t(float a, float b) {
  // keep sign, 8-bit exponent and top 7 mantissa bits of each float32 word
  return (__float_as_uint(a) >> 16) | (__float_as_uint(b) & 0xffff0000u);
}
__device__ __forceinline__ uint4 pack(df_t, const dfl* r) {
  return make_uint4(__float_as_uint(r[0].hi), __float_as_uint(r[0].lo), __float_as_uint(r[1].hi),
                    __float_as_uint(r[1].lo));
}
__device__ __forceinline__ uint4 pack(f16_t, const float* r) {
  return make_uint4(f2h2(r[0], r[1]), f2h2(r[2], r[3]), f2h2(r[4], r[5]), f2h2(r[6], r[7]));
}
__device__ __forceinline__ uint4 pack(bf16_t, const float* r) {
  return make_uint4(f2b2(r[0], r[1]), f2b2(r[2], r[3]), f2b2(r[4], r[5]), f2b2(r[6], r[7]));
}
__device__ __forceinline__ uint4 pack(bf16t_t, const float* r) {
  return make_uint4(f2b2t(r[0], r[1]), f2b2t(r[2], r[3]), f2b2t(r[4], r[5]), f2b2t(r[6], r[7]));
}

// whole-spinor load / store in the chunked layout ------------------------------
template <typename St, typename R>
__device__ __forceinline__ void load_spinor(const uint4* __restrict__ f, size_t site5, size_t n5,
                                            R* v) {
  constexpr int C = Store<St>::chunks, P = Store<St>::per_chunk;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    uint4 g = __ldg(f + c * n5 + site5);
    typename Store<St>::real t[P];
    unpack(St{}, g, t);
#pragma unroll
    for (int i = 0; i < P; ++i) v[c * P + i] = (R)t[i];
  }
}

template <typename St, typename R>
__device__ __forceinline__ void store_spinor(uint4* __restrict__ f, size_t site5, size_t n5,
                                             const R* v) {
  constexpr int C = Store<St>::chunks, P = Store<St>::per_chunk;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    typename Store<St>::real t[P];
#pragma unroll
    for (int i = 0; i < P; ++i) t[i] = (typename Store<St>::real)v[c * P + i];
    f[c * n5 + site5] = pack(St{}, t);
  }
}

// deterministic FP64 reductions ---------------------------------------------------
// Each block writes NV partial sums to partials[NV * blockIdx.x + i]; the last
// block to finish (atomic ticket) sums the partials in a fixed order and stores
// the totals to result[i] (optionally accumulating), then resets the ticket.
//
// Multi-right-hand-side kernels reduce NV = k * RED_RHS values laid out as k
// groups of RED_RHS slots; with `active` right-hand sides, slots whose index
// modulo RED_RHS is >= active are known to be zero and are skipped (their
// totals are written as zero).  FP64 adds are slow on GB300, so a reduction
// of 16 or 32 slots for one right-hand side would otherwise dominate small
// kernels.
constexpr int RED_RHS = 16;   // equals RMAX, the right-hand sides per batch

template <int NV>
__device__ __forceinline__ bool red_active(int i, int active) {
  return NV < RED_RHS || (i % RED_RHS) < active;
}

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV], int active = RED_RHS) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (red_active<NV>(i, active)) v[i] += __shfl_xor_sync(FULL_MASK, v[i], o);
}

// PRE: the values are already summed over each warp (valid in lane 0)
template <int NV, bool PRE = false>
__device__ void block_sum(double (&v)[NV], int active = RED_RHS) {
  __shared__ double sh[32][NV];
  if (!PRE) warp_sum<NV>(v, active);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[w][i] = v[i];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = lane < nw ? sh[lane][i] : 0.0;
    warp_sum<NV>(v, active);
  }
}

// Several right-hand sides reduce independently: the grid's y index selects
// the right-hand side (its own partials, ticket and result, result_stride
// doubles apart); one right-hand side is gridDim.y = 1.
struct Reduction {
  double* partials;     // >= NV * gridDim.x * gridDim.y doubles
  unsigned* ticket;     // gridDim.y tickets, zero between uses
  double* result;       // NV doubles per right-hand side
  int accumulate;       // 1: result += total, 0: result = total
  int result_stride;    // doubles between the results of consecutive right-hand sides
};

// Returns true in every thread of the last block (after the totals are stored).
// PRE: v already holds per-warp sums in lane 0 (see block_sum).
template <int NV, bool PRE = false>
__device__ bool grid_reduce(double (&v)[NV], const Reduction& red, int active = RED_RHS) {
  block_sum<NV, PRE>(v, active);
  __shared__ bool last;
  const unsigned y = blockIdx.y;
  double* partials = red.partials + (size_t)NV * gridDim.x * y;
  unsigned* ticket = red.ticket + y;
  double* result = red.result + (size_t)red.result_stride * y;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[NV * blockIdx.x + i] = v[i];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (red_active<NV>(i, active)) acc[i] += ((volatile double*)partials)[NV * b + i];
  block_sum<NV>(acc, active);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) result[i] = red.accumulate ? result[i] + acc[i] : acc[i];
    *ticket = 0;
  }
  return true;
}

}  // namespace hdcg
